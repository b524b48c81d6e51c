"""The k trade-off of the superposition approximation (Sec. 4.1, the paper's
relative-error-versus-k study) on the GPU.

For a fixed problem, sweep k over four decades and measure, against the FP64
oracle: the FP32 error at the same k (falls like 1/k: cancellation against
the FP32 time-reversal error of u^s) and the approximation gap to the exact
gradient (grows like k: the neglected k^2 K(u_adj, u_adj) of Eq.
superposedkernel1).  The test checks those two trends and that a band of k
exists where the total FP32 error is below 5% (the paper's threshold).
"""
import numpy as np
import pytest

import oracle as O
from _problems import make_problem, rel_l2

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2509_15744_gb300 import wave
    return wave


def test_k_sweep_velocity_l2(W):
    prob = make_problem((128, 128), 2, "dirichlet", nt=400, nrec=64, seed=5)
    med = prob.medium()
    shots = prob.oracle_shots()
    _, g_exact, _ = O.exact_gradient(med, shots, 400)
    m = W.Model(torch.from_numpy(prob.param0).to(DEV), prob.h, prob.dt, 2, "velocity", "dirichlet")
    wav = W.wavelet(prob.wav_kind, prob.wav_freq, prob.dt, 400, device=DEV)
    shot = W.Shot(prob.src[0], wav, torch.from_numpy(prob.rec[0]).to(DEV),
                  torch.from_numpy(prob.observed[0]).to(DEV))
    rows = []
    for r in (1e-4, 1e-3, 1e-2, 1e-1):
        g, _, kd = m.gradient([shot], k_ratio=r)
        torch.cuda.synchronize()
        k = float(kd.item())
        sup = O.superposition_gradient(med, shots, 400, k)
        gg = g.cpu().numpy()
        rows.append((r, rel_l2(gg, sup["K_tilde"]), rel_l2(sup["K_tilde"], g_exact), rel_l2(gg, g_exact)))
    print("\n  k_ratio   fp32-vs-oracle   gap(fp64)   total(fp32)")
    for r, e32, gap, tot in rows:
        print(f"  {r:7.0e}   {e32:14.2e}   {gap:9.2e}   {tot:11.2e}")
    e32 = [x[1] for x in rows]
    gaps = [x[2] for x in rows]
    assert all(a > b for a, b in zip(e32, e32[1:]))          # FP32 error falls with k
    assert all(a < b for a, b in zip(gaps, gaps[1:]))        # approximation gap grows with k
    assert min(x[3] for x in rows) < 0.05                    # a usable band exists
    # the FP32 error scales about as 1/k and the gap about as k
    assert 3 < e32[0] / e32[1] < 30 and 3 < gaps[1] / gaps[0] < 30
