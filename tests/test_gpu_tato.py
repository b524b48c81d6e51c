"""The topology-optimisation design chain on the GPU (Sec. 5.2, Sec. 6.2): the
gradient of C(design(gamma)) with respect to gamma through torch autograd and
libwave's sensitivity, against the oracle's exact gradient at the same design
chain-ruled in FP64; and a short Adam run that lowers the patch energy."""
import numpy as np
import pytest

import oracle as O
from _problems import make_problem, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2509_15744_gb300 import autograd, tato, wave
    return wave, autograd, tato


def patch_problem():
    shape = (60, 150)
    ny, nx = shape
    py, px = np.meshgrid(np.arange(20, 40), np.arange(120, 150), indexing="ij")
    patch = (py * nx + px).ravel()
    return make_problem(shape, physics="density", bc="neumann", nt=300, objective="patch", patch=patch,
                        src=ny // 2 * nx + 60, seed=3, patch_sign=1.0)


def gpu_problem(W, A, prob, **kw):
    wav = W.wavelet(prob.wav_kind, prob.wav_freq, prob.dt, prob.nt[0], device=DEV)
    shots = [W.Shot(prob.src[0], wav, torch.from_numpy(prob.rec[0]).to(DEV), None)]
    return A.WaveProblem(h=prob.h, dt=prob.dt, shots=shots, order=2, physics="density", bc="neumann",
                         objective="patch", patch_sign=1.0, **kw)


def test_design_chain_gradient_matches_oracle(env):
    W, A, T = env
    prob = patch_problem()
    rf, beta = 1.5, 1.1 ** 3
    gamma32 = torch.nn.Parameter(torch.from_numpy(prob.param0).to(DEV))
    problem = gpu_problem(W, A, prob, mode="symmetric", k_ratio=0.1)
    c = A.wave_misfit(T.design(gamma32, rf, beta).contiguous(), problem)
    c.backward()
    g_gpu = gamma32.grad.detach().cpu().numpy()
    # oracle: exact gradient at the FP64 design, chain-ruled through the same map in FP64
    gamma64 = torch.from_numpy(prob.param0.astype(np.float64)).requires_grad_(True)
    d64 = T.design(gamma64, rf, beta)
    med = O.Medium("density", d64.detach().numpy(), prob.h, prob.dt, 2, "neumann")
    c_ref, g_design, _ = O.exact_gradient(med, prob.oracle_shots(), prob.nt[0])
    (d64 * torch.from_numpy(g_design)).sum().backward()
    g_ref = gamma64.grad.numpy()
    err = rel_l2(g_gpu, g_ref)
    print(f"\ndesign-chain gradient vs oracle: {err:.2e}")
    assert err < 1e-3
    assert abs(float(c.item()) - c_ref) < 1e-5 * abs(c_ref)


def test_short_adam_run_lowers_the_patch_energy(env):
    W, A, T = env
    prob = patch_problem()
    problem = gpu_problem(W, A, prob, mode="symmetric", k_ratio=0.1)
    gamma0 = torch.from_numpy(prob.param0).to(DEV)
    gamma, hist = T.optimise(gamma0, problem, iterations=8, lr=0.1)
    print("\npatch energy over 8 Adam iterations: " + ", ".join(f"{h:.3e}" for h in hist))
    assert hist[-1] < 0.9 * hist[0]
    assert float(gamma.min()) >= float(np.float32(1e-5)) and float(gamma.max()) <= 1.0   # clip bounds in FP32
    d = T.design(gamma, 1.5, T.beta_schedule(7))
    assert float(d.min()) >= 0.0 and float(d.max()) <= 1.0
