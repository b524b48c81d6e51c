"""One leapfrog step of several fields through wave_step (the step of
Algorithm 1's loops, Eq. FDstencil1 / FDstencil2 without force), from seeded
random levels, against the oracle's step and sensitivity increment on the
whole grid.  3D velocity fields with FP32 storage run in one launch (the
batched gradient's configuration); the rest run one launch per field.
"""
import numpy as np
import pytest

import oracle as O
from _problems import rel_l2

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


def pitched(a: np.ndarray, px: int, dtype=torch.float32) -> torch.Tensor:
    out = np.zeros(a.shape[:-1] + (px,), np.float32)
    out[..., : a.shape[-1]] = a
    return torch.from_numpy(out).to(DEV).to(dtype)


def dense(t: torch.Tensor, nx: int) -> np.ndarray:
    return t.float().cpu().numpy()[..., :nx].astype(np.float64)


def oracle_increment(med: O.Medium, u: np.ndarray, u_new: np.ndarray) -> np.ndarray:
    # sensitivity increment of one step in the accumulator's units (-dt times
    # the discrete kernel): the half-level term of (u^{n+1} - u^n) and, for the
    # density form, the level term of u^n
    d = u_new - u
    return -med.dt * (med.kernel_half_level(d, d) + med.kernel_level(u, u))


CASES = [
    ("vel3d_o8_dirichlet", (19, 21, 133), "velocity", 8, "dirichlet", "f32"),
    ("vel3d_o4_neumann", (12, 17, 260), "velocity", 4, "neumann", "f32"),
    ("vel2d_o6_neumann", (37, 141), "velocity", 6, "neumann", "f32"),
    ("dens2d_neumann", (30, 150), "density", 2, "neumann", "f32"),
    ("dens3d_dirichlet", (9, 11, 131), "density", 2, "dirichlet", "f32"),
    ("vel3d_o8_bf16", (11, 13, 140), "velocity", 8, "dirichlet", "bf16"),
]


@pytest.mark.parametrize("kahan", [False, True])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_step_of_several_fields_matches_oracle(W, case, kahan):
    name, shape, physics, order, bc, storage = case
    rng = np.random.default_rng(71)
    if physics == "velocity":
        param = rng.uniform(1500.0, 4500.0, shape).astype(np.float32)
        h = 10.0
        dt = O.cfl_dt(h, 4500.0, len(shape), order, 0.5)
    else:
        param = rng.uniform(0.1, 1.0, shape).astype(np.float32)
        h = 2e-3
        dt = O.cfl_dt(h, 509.8366, len(shape), 2, 0.5)
    nf = 3
    signs = [1.0, -1.0, 0.5]
    lvl = [rng.standard_normal((2,) + shape).astype(np.float32) for _ in range(nf)]
    if storage == "bf16":   # the oracle starts from the stored (rounded) values
        lvl = [torch.from_numpy(x).to(torch.bfloat16).float().numpy() for x in lvl]
    m = W.Model(torch.from_numpy(param).to(DEV), h, dt, order, physics, bc, storage=storage, kahan=kahan)
    px = m.pitch
    assert px % 128 == 0 and px >= shape[-1]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    cur = [pitched(x[1], px, tdt) for x in lvl]
    prev = [pitched(x[0], px, tdt) for x in lvl]
    acc0 = rng.standard_normal(shape).astype(np.float32)
    acc = pitched(acc0, px)
    comp = pitched(np.zeros(shape, np.float32), px) if kahan else None
    m.step(cur, prev, acc=acc, comp=comp, acc_sign=signs)
    torch.cuda.synchronize()
    med = O.Medium(physics, param.astype(np.float64), h, dt, order, bc)
    acc_ref = acc0.astype(np.float64)
    tol = 1e-5 if storage == "f32" else 1e-2
    for f in range(nf):
        u_prev, u = lvl[f][0].astype(np.float64), lvl[f][1].astype(np.float64)
        u_new = med.step(u_prev, u, np.zeros(shape))
        got = dense(prev[f], shape[-1])
        assert rel_l2(got, u_new) < tol, (f, rel_l2(got, u_new))
        # sensitivity increment of Algorithm 1 with the level the kernel stored
        acc_ref += signs[f] * oracle_increment(med, u, got if storage == "bf16" else u_new)
        # padding stays zero
        assert float(prev[f].float()[..., shape[-1]:].abs().max()) == 0.0
    got_acc = dense(acc, shape[-1])
    assert rel_l2(got_acc, acc_ref) < (1e-5 if storage == "f32" else 1e-3)
    assert float(acc[..., shape[-1]:].abs().max()) == 0.0


def test_step_without_accumulator_and_argument_checks(W):
    shape = (10, 12, 130)
    rng = np.random.default_rng(72)
    param = rng.uniform(1500.0, 4500.0, shape).astype(np.float32)
    dt = O.cfl_dt(10.0, 4500.0, 3, 4, 0.5)
    m = W.Model(torch.from_numpy(param).to(DEV), 10.0, dt, 4, "velocity", "dirichlet")
    px = m.pitch
    lv = rng.standard_normal((2,) + shape).astype(np.float32)
    cur, prev = pitched(lv[1], px), pitched(lv[0], px)
    m.step([cur], [prev])
    torch.cuda.synchronize()
    med = O.Medium("velocity", param.astype(np.float64), 10.0, dt, 4, "dirichlet")
    ref = med.step(lv[0].astype(np.float64), lv[1].astype(np.float64), np.zeros(shape))
    assert rel_l2(dense(prev, shape[-1]), ref) < 1e-5
    with pytest.raises(ValueError):
        m.step([cur], [torch.zeros(shape[:-1] + (px - 1,), device=DEV)])
    with pytest.raises(W.WaveError):          # the same buffer as both levels
        m.step([cur], [cur])
