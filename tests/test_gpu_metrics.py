"""Per-call figures of the gradient call: the FP64 gradient norm of the finish
pass, the metrics record (misfit, k, per-pass device times, algorithmic
bytes, cell-updates), new parameters for an existing model, and the
non-finite checks (a NaN parameter, NaN data), all fed from the host."""
import numpy as np
import pytest
import torch

import oracle as O
from _gpu import gpu_model, gpu_shots
from _problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as ge
    ge.build()
    from paper_2509_15744_gb300 import wave
    return wave


@pytest.mark.parametrize("shape,order,batched,mode", [((48, 150), 4, False, "superposition"),
                                                      ((14, 20, 133), 8, True, "superposition"),
                                                      ((14, 20, 133), 8, False, "reverse"),
                                                      ((40, 90), 2, False, "exact")])
def test_gradient_norm_is_the_fp64_norm_of_the_result(W, shape, order, batched, mode):
    nsh = 3 if batched else 1
    prob = make_problem(shape, order, "dirichlet", nshots=nsh, nt_list=[40, 33, 37][:nsh], nrec=30, seed=81)
    m = gpu_model(W, prob)
    g, c, k = m.gradient(gpu_shots(W, prob), batched=batched, mode=mode)
    torch.cuda.synchronize()
    got = float(m.grad_norm.item())
    ref = float(np.linalg.norm(g.cpu().numpy().astype(np.float64)))
    assert abs(got - ref) <= 1e-12 * ref                      # the reduction itself
    if mode == "superposition":
        kt = sum(O.superposition_gradient(prob.medium(), [s], n, float(k.item()))["K_tilde"]
                 for s, n in zip(prob.oracle_shots(), prob.nt))
        assert abs(got - np.linalg.norm(kt)) <= 1e-3 * np.linalg.norm(kt)   # within the K~ parity bar


@pytest.mark.parametrize("batched", [False, True])
def test_metrics_record_of_a_call(W, batched):
    shape, nts = (20, 24, 140), [30, 22, 26]
    prob = make_problem(shape, 8, "dirichlet", nshots=3, nt_list=nts, nrec=30, seed=82)
    m = gpu_model(W, prob)
    m.set_metrics(True)
    g, c, k = m.gradient(gpu_shots(W, prob), batched=batched)
    rec = m.metrics()
    assert rec["misfit"] == float(c.item())
    assert rec["k"] == float(k.item())
    assert rec["grad_l2"] == pytest.approx(float(m.grad_norm.item()), rel=1e-15)
    cells = int(np.prod(shape))
    assert rec["cell_updates"] == cells * sum(nts)
    # step launches: one per global step and pass (batched) or per shot, step and pass
    launches = 2 * max(nts) if batched else 2 * sum(nts)
    assert rec["step_launches"] == launches
    if not batched:   # 12 B per cell (u^n, u^{n-1}, coef, u^{n+1}) + 8 B accumulator where it accumulates
        acc_launches = sum(2 * n - 1 for n in nts)
        assert rec["step_bytes"] == pytest.approx(cells * (16.0 * launches + 8.0 * acc_launches))
    assert rec["forward_ms"] > 0 and rec["adjoint_ms"] > 0
    assert rec["forward_ms"] + rec["adjoint_ms"] <= rec["total_ms"] * (1 + 1e-6)
    m.set_metrics(False)
    with pytest.raises(W.WaveError):
        m.metrics()


def test_new_parameter_for_an_existing_model(W):
    prob = make_problem((30, 140), 4, "dirichlet", nt=50, nrec=30, seed=83)
    m = gpu_model(W, prob)
    g0, _, _ = m.gradient(gpu_shots(W, prob), k=1.0)
    p2 = prob.param0 * np.float32(1.05)
    m.set_param(torch.from_numpy(np.ascontiguousarray(p2)).cuda())
    g1, c1, _ = m.gradient(gpu_shots(W, prob), k=1.0)
    fresh = gpu_model(W, prob, param=p2)
    g2, c2, _ = fresh.gradient(gpu_shots(W, prob), k=1.0)
    torch.cuda.synchronize()
    assert m.check() == 0
    assert torch.equal(g1, g2) and float(c1.item()) == float(c2.item())
    assert not torch.equal(g0, g1)
    # an unstable velocity and a NaN are reported by check(), not by a fault
    m.set_param(torch.from_numpy(np.ascontiguousarray(prob.param0 * np.float32(3.0))).cuda())
    assert m.check() == 2
    bad = prob.param0.copy()
    bad[3, 7] = np.nan
    m.set_param(torch.from_numpy(bad).cuda())
    assert m.check() == 6


def test_non_finite_inputs_are_reported(W):
    prob = make_problem((30, 140), 4, "dirichlet", nt=40, nrec=30, seed=84)
    bad = prob.param0.copy()
    bad[5, 5] = np.inf
    with pytest.raises(W.WaveError) as e:
        gpu_model(W, prob, param=bad)
    assert e.value.status == 6
    m = gpu_model(W, prob)
    m.set_metrics(True)
    shots = gpu_shots(W, prob)
    shots[0].observed[2, 10] = float("nan")
    m.gradient(shots, k=1.0)
    with pytest.raises(W.WaveError) as e:
        m.metrics()
    assert e.value.status == 6
    # the model stays usable
    g, _, _ = m.gradient(gpu_shots(W, prob), k=1.0)
    m.metrics()
    assert torch.isfinite(g).all()


def test_workspace_too_small_or_misaligned_is_refused(W):
    prob = make_problem((20, 24, 140), 4, "dirichlet", nshots=2, nt_list=[10, 8], nrec=20, seed=85)
    m = gpu_model(W, prob)
    shots = gpu_shots(W, prob)
    arr = W._shot_descs(shots)
    o = W.GradOpts()
    o.objective, o.mode, o.batched, o.grad_wrt = 0, 0, 1, 0
    o.k = 1.0
    need = W._sz(0)
    assert W._grad_ws(m._h, arr, len(shots), W.C.byref(o), W.C.byref(need)) == 0
    ws = torch.empty(need.value + 512, dtype=torch.uint8, device="cuda")
    grad = torch.empty(prob.shape, dtype=torch.float32, device="cuda")
    st = W._stream()

    def call(ptr, size):
        return W._adjoint_sensitivity(m._h, arr, len(shots), W.C.byref(o), W._ptr(grad), None, None, None,
                                      W.C.c_void_p(ptr), size, st)
    assert call(ws.data_ptr(), need.value - 1) == 3
    assert call(ws.data_ptr() + 64, need.value) == 3
    assert call(ws.data_ptr(), need.value) == 0
    torch.cuda.synchronize()
    traces = [torch.empty((s.nrec, s.nt + 1), dtype=torch.float32, device="cuda") for s in shots]
    farr = W._shot_descs(shots, traces)
    fws = W._sz(0)
    assert W._fwd_ws(m._h, farr, len(shots), W.C.byref(fws)) == 0
    assert W._forward(m._h, farr, len(shots), None, None, W.C.c_void_p(ws.data_ptr()), fws.value - 1, st) == 3
    assert W._forward(m._h, farr, len(shots), None, None, W.C.c_void_p(ws.data_ptr() + 16), fws.value, st) == 3
