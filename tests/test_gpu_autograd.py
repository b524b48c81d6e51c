"""torch.autograd.Function over the CUDA path: gradient checks.

* velocity: the autograd gradient equals the oracle's superposition
  gradient chain-ruled to dC/dv (same k, parity bar 1e-3), stays within the
  approximation gap of the exact adjoint gradient, and matches central finite
  differences of the GPU misfit;
* density (a 64^2 crop of the topology-optimisation workload, patch energy):
  against central finite differences of the FP64 oracle misfit.
"""
import numpy as np
import pytest

import oracle as O
from _problems import make_problem, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2509_15744_gb300 import autograd as A
    from paper_2509_15744_gb300 import wave as W
    return W, A


def _gpu_shots(W, prob):
    out = []
    for i in range(len(prob.src)):
        wav = W.wavelet(prob.wav_kind, prob.wav_freq, prob.dt, prob.nt[i], device=DEV)
        obs = None if prob.observed is None else torch.from_numpy(prob.observed[i]).to(DEV)
        out.append(W.Shot(prob.src[i], wav, torch.from_numpy(prob.rec[i]).to(DEV), obs))
    return out


def test_velocity_autograd_against_oracle_and_fd(mods):
    W, A = mods
    prob = make_problem((40, 130), order=4, bc="dirichlet", nt=160, nrec=40, seed=31)
    pb = A.WaveProblem(h=prob.h, dt=prob.dt, shots=_gpu_shots(W, prob), order=4, bc="dirichlet")
    v = torch.from_numpy(prob.param0).to(DEV).requires_grad_(True)
    c = A.wave_misfit(v, pb)
    c.backward()
    g = v.grad.cpu().numpy().astype(np.float64)
    k = float(pb.last_k.item())
    med = prob.medium()
    shots = prob.oracle_shots()
    sup = O.superposition_gradient(med, shots, prob.nt[0], k)
    assert abs(float(c.item()) - sup["C"]) < 1e-5 * sup["C"]
    assert rel_l2(g, med.param_chain(sup["K_tilde"])) < 1e-3
    _, g_exact, _ = O.exact_gradient(med, shots, prob.nt[0])
    gap = rel_l2(g, med.param_chain(g_exact))
    print(f"\nautograd dC/dv: gap to exact adjoint {gap:.2e}")
    assert gap < 0.05
    # central finite differences of the GPU misfit along a random direction
    rng = np.random.default_rng(3)
    d = torch.from_numpy(rng.standard_normal(prob.param0.shape).astype(np.float32)).to(DEV)
    eps = 2.0
    with torch.no_grad():
        cp = A.wave_misfit(v.detach() + eps * d, pb)
        cm = A.wave_misfit(v.detach() - eps * d, pb)
    fd = (float(cp.item()) - float(cm.item())) / (2 * eps)
    an = float((v.grad * d).sum().item())
    print(f"autograd dC/dv: FD {fd:.6e} vs gradient {an:.6e}")
    assert abs(fd - an) < 0.05 * abs(fd)


def test_density_autograd_against_finite_differences(mods):
    W, A = mods
    from paper_2509_15744_gb300 import workloads as WL
    n = 64
    w3 = WL.workload3(n=256)
    gamma = np.ascontiguousarray(np.asarray(w3.init_param)[:n, :n])
    py, px = np.meshgrid(np.arange(24, 40), np.arange(54, 64), indexing="ij")
    patch = (py * n + px).ravel().astype(np.int64)
    src = 32 * n + 2
    h = w3.h
    dt = O.cfl_dt(h, w3.vmax, 2, 2, 0.5)
    nt = 300
    freq = 1.0 / (30 * dt)
    wav_d = W.wavelet("sine_burst", freq, dt, nt, device=DEV)
    shot = W.Shot(src, wav_d, torch.from_numpy(patch).to(DEV))
    wav = O.sine_burst(np.arange(nt + 1) * dt, freq, 2, 1.0)
    oshot = O.Shot(src, wav, patch, None, O.patch_weight(len(patch), 1.0))
    med = O.Medium("density", gamma.astype(np.float64), h, dt, 2, "neumann")
    # (1) parity with the oracle at the same k, where FP32 cancellation is
    # below the bar (k u_adj / u large enough)
    pb = A.WaveProblem(h=h, dt=dt, shots=[shot], order=2, physics="density", bc="neumann", objective="patch",
                       k_ratio=5e-2)
    gm = torch.from_numpy(gamma).to(DEV).requires_grad_(True)
    A.wave_misfit(gm, pb).backward()
    sup = O.superposition_gradient(med, [oshot], nt, float(pb.last_k.item()))
    assert rel_l2(gm.grad.cpu().numpy(), sup["K_tilde"]) < 1e-3
    # (2) the gradient near the best k against FP64 finite differences.  For
    # this strongly scattering random medium and a patch far from the source,
    # the approximation gap grows with k and the FP32 time-reversal error falls
    # as 1/k; their best sum is about 10% (measured on GB300 over a k sweep),
    # so the finite-difference check is held to 25%.
    pb = A.WaveProblem(h=h, dt=dt, shots=[shot], order=2, physics="density", bc="neumann", objective="patch",
                       k_ratio=1e-4, kahan=True)
    gm = torch.from_numpy(gamma).to(DEV).requires_grad_(True)
    c = A.wave_misfit(gm, pb)
    c.backward()
    g = gm.grad.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((n, n))
    eps = 1e-4

    def cost(gam):
        m2 = O.Medium("density", gam, h, dt, 2, "neumann")
        tr = O.forward(m2, oshot, nt)["traces"]
        return O.misfit(tr, None, dt, oshot.weight)

    fd = (cost(gamma + eps * d) - cost(gamma - eps * d)) / (2 * eps)
    an = float(np.sum(g * d))
    print(f"\ndensity autograd (patch): FD {fd:.6e} vs gradient {an:.6e}")
    assert abs(fd - an) < 0.25 * abs(fd)


def test_density_l2_autograd_against_finite_differences(mods):
    W, A = mods
    prob = make_problem((48, 140), physics="density", bc="neumann", nt=220, nrec=60, seed=33)
    pb = A.WaveProblem(h=prob.h, dt=prob.dt, shots=_gpu_shots(W, prob), order=2, physics="density",
                       bc="neumann", k_ratio=1e-2)
    gm = torch.from_numpy(prob.param0).to(DEV).requires_grad_(True)
    A.wave_misfit(gm, pb).backward()
    g = gm.grad.cpu().numpy().astype(np.float64)
    shots = prob.oracle_shots()
    rng = np.random.default_rng(6)
    d = rng.standard_normal(prob.param0.shape)
    eps = 1e-4

    def cost(gam):
        m2 = O.Medium("density", gam, prob.h, prob.dt, 2, "neumann")
        tr = O.forward(m2, shots[0], prob.nt[0])["traces"]
        return O.misfit(tr, shots[0].observed, prob.dt)

    p0 = prob.param0.astype(np.float64)
    fd = (cost(p0 + eps * d) - cost(p0 - eps * d)) / (2 * eps)
    an = float(np.sum(g * d))
    print(f"\ndensity autograd (L2): FD {fd:.6e} vs gradient {an:.6e}")
    assert abs(fd - an) < 0.05 * abs(fd)
