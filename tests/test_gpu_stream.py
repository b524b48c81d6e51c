"""The TMA-tiled batched step kernel (tiling pipeline 5): the shots of a
launch one after the other over z-blocks of 8 planes, the accumulator of the
block in registers across them.

It performs the arithmetic of the other 3D pipelines element by element, so
its results must be bit-identical to the two-shots-per-pass kernel, which the
oracle parity tests pin.  The shapes put CTAs at every kind of edge: y
boundaries at both ends and interior row tiles (ny = 50), partial last
z-blocks (nz not a multiple of 8, one plane in the last block), ragged x
strips (nx = 261) and strip-aligned rows, odd and even shot counts, uneven
record lengths, both boundary conditions, all four orders, Kahan on and off;
the exact reverse-time mode under this tiling (its (u, lambda) launches go to
the two-shots-per-pass kernel) gives the same result too.
"""
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


@pytest.mark.parametrize("order,bc,shape,nts,kahan", [
    (8, "dirichlet", (29, 50, 261), [14, 9, 12], False),
    (8, "neumann", (29, 50, 261), [14, 9, 12, 11], True),
    (6, "dirichlet", (17, 19, 130), [10, 7], False),
    (4, "neumann", (12, 40, 133), [9, 9, 8, 6, 7], False),
    (2, "dirichlet", (9, 21, 259), [8, 5, 6], True),
    (2, "neumann", (9, 21, 259), [8, 5, 6], False),
])
def test_stream_pipeline_matches_pair_kernel_bitwise(W, order, bc, shape, nts, kahan):
    prob = make_problem(shape, order, bc, nshots=len(nts), nt_list=nts, nrec=40, seed=71)
    m = gpu_model(W, prob, kahan=kahan)
    m.set_tiling(16, 16, 2, 4)
    g4, c4, _ = m.gradient(gpu_shots(W, prob), batched=True, k=1.5)
    r4, _, _ = m.gradient(gpu_shots(W, prob)[:1], mode="reverse")
    torch.cuda.synchronize()
    for depth in (2, 3):
        m.set_tiling(8, 16, depth, 5)
        g5, c5, _ = m.gradient(gpu_shots(W, prob), batched=True, k=1.5)
        r5, _, _ = m.gradient(gpu_shots(W, prob)[:1], mode="reverse")
        torch.cuda.synchronize()
        assert m.check() == 0
        assert torch.equal(g5, g4)
        assert float(c5.item()) == float(c4.item())
        assert torch.equal(r5, r4)


def test_stream_pipeline_one_step_of_many_fields_matches_oracle(W):
    # wave_step with 5 fields (passes of 2, 2, 1) against the oracle's step and
    # the signed increments, on a grid with interior and boundary row tiles
    rng = np.random.default_rng(3)
    shape, order, bc = (19, 52, 140), 8, "dirichlet"
    v = rng.uniform(1500, 4500, shape).astype(np.float32)
    dt = O.cfl_dt(10.0, 4500.0, 3, order, 0.5)
    m = W.Model(torch.from_numpy(v).cuda(), 10.0, dt, order, "velocity", bc)
    m.set_tiling(8, 16, 2, 5)
    px = m.pitch
    nf = 5
    cur = [rng.standard_normal(shape).astype(np.float32) for _ in range(nf)]
    prev = [rng.standard_normal(shape).astype(np.float32) for _ in range(nf)]
    sign = [1.0, -1.0, 0.5, 0.0, 2.0]

    def pitched(a):
        out = np.zeros(shape[:-1] + (px,), np.float32)
        out[..., :shape[-1]] = a
        return torch.from_numpy(out).cuda()
    cd = [pitched(a) for a in cur]
    pd = [pitched(a) for a in prev]
    acc = torch.zeros(shape[:-1] + (px,), dtype=torch.float32, device="cuda")
    m.step(cd, pd, acc=acc, acc_sign=sign)
    torch.cuda.synchronize()
    assert m.check() == 0
    med = O.Medium("velocity", v.astype(np.float64), 10.0, dt, order, bc)
    inc = np.zeros(shape)
    for f in range(nf):
        ref = med.step(prev[f].astype(np.float64), cur[f].astype(np.float64), np.zeros(shape))
        got = pd[f].cpu().numpy()[..., :shape[-1]]
        assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
        inc += sign[f] * (ref - cur[f]) ** 2
        assert not pd[f].cpu().numpy()[..., shape[-1]:].any()   # padding stays zero
    assert rel_l2(acc.cpu().numpy()[..., :shape[-1]], inc) < 1e-5


def test_stream_pipeline_wait_times_out_without_hanging(W):
    # Failure detection: with the copies switched off every bounded wait runs
    # out; the call reports WAVE_ETIMEOUT and the context stays usable.
    prob = make_problem((20, 40, 140), 4, "dirichlet", nshots=2, nt_list=[6, 5], nrec=10, seed=62)
    m = gpu_model(W, prob)
    m.set_tiling(8, 16, 2, 5)
    ref, _, _ = m.gradient(gpu_shots(W, prob), batched=True, k=1.0)
    torch.cuda.synchronize()
    assert m.check() == 0
    m.set_debug(True, wait_limit_cycles=2_000_000)
    m.gradient(gpu_shots(W, prob), batched=True, k=1.0)
    assert m.check() == 5
    m.set_debug(False)
    again, _, _ = m.gradient(gpu_shots(W, prob), batched=True, k=1.0)
    torch.cuda.synchronize()
    assert m.check() == 0
    assert torch.equal(again, ref)
