"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
discrete solutions, invariants of the leapfrog scheme, adjoint identities,
finite differences, and values the paper prints.  A plausible mistake in the
oracle (a dropped term, a wrong sign or index, a transposed operand) breaks at
least one of them; test_planted_mistakes checks that on purpose.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Stencil weights: Taylor conditions solved exactly, polynomial exactness
# ---------------------------------------------------------------------------
def _taylor_second_derivative_weights(order):
    """Solve sum_j w_j j^(2q) = 2 [q == 1] / ... for symmetric weights.

    Symmetric weights w_0, w_1..w_r (w_-j = w_j) of d^2/dx^2 satisfy, for the
    Taylor moments, w_0 + 2 sum w_j = 0 and 2 sum_j w_j j^(2q) / (2q)! = [q==1]
    for q = 1..r.  Solved here with exact rational Gaussian elimination.
    """
    r = order // 2
    n = r + 1
    rows = []
    rhs = []
    rows.append([Fraction(1)] + [Fraction(2)] * r)
    rhs.append(Fraction(0))
    for q in range(1, r + 1):
        rows.append([Fraction(0)] + [Fraction(2 * j ** (2 * q), math.factorial(2 * q)) for j in range(1, r + 1)])
        rhs.append(Fraction(1 if q == 1 else 0))
    a = [row[:] + [b] for row, b in zip(rows, rhs)]
    for col in range(n):
        piv = next(i for i in range(col, n) if a[i][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        for i in range(n):
            if i != col and a[i][col] != 0:
                f = a[i][col] / a[col][col]
                a[i] = [x - f * y for x, y in zip(a[i], a[col])]
    return tuple(a[i][n] / a[i][i] for i in range(n))


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_weights_solve_taylor_conditions(order):
    assert _taylor_second_derivative_weights(order) == O.SECOND_DERIVATIVE_WEIGHTS[order]


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_laplacian_exact_on_polynomials(order):
    # The order-p central second derivative is exact for polynomials of degree
    # <= p + 1; away from the boundary the ghost cells play no role.
    r = order // 2
    h = 0.37
    n = 4 * r + 9
    x = (np.arange(n) - n // 2) * h
    for p in range(0, order + 2):
        u = x ** p
        d2 = p * (p - 1) * x ** (p - 2) if p >= 2 else np.zeros(n)
        lu = O.laplacian(u, h, order, "neumann")
        inner = slice(r, n - r)
        np.testing.assert_allclose(lu[inner], d2[inner], rtol=1e-9, atol=1e-7 * (1 + np.abs(d2[inner]).max()))
    # and not exact for degree p + 2 (so the order is not higher than claimed)
    u = x ** (order + 2)
    d2 = (order + 2) * (order + 1) * x ** order
    lu = O.laplacian(u, h, order, "neumann")
    assert np.abs(lu[r:n - r] - d2[r:n - r]).max() > 1e-6


def test_truncation_order_under_refinement():
    # Error of the order-p Laplacian on sin(x) decreases like h^p.
    for order in (2, 4, 6, 8):
        errs = []
        for n in (6, 12):
            h = 1.0 / n
            x = np.arange(6 * n) * h
            u = np.sin(2.0 * x)
            lu = O.laplacian(u, h, order, "neumann")
            r = order // 2
            errs.append(np.abs(lu[r:-r] + 4.0 * u[r:-r]).max())
        rate = math.log2(errs[0] / errs[1])
        assert abs(rate - order) < 0.35, (order, rate)


def test_symbol_maximum_matches_numeric_supremum():
    theta = np.linspace(0.0, np.pi, 200001)
    for order in (2, 4, 6, 8):
        c = O.stencil_weights(order)
        sym = c[0] + 2 * sum(c[j] * np.cos(j * theta) for j in range(1, len(c)))
        assert abs(np.abs(sym).max() - O.stencil_symbol_max(order)) < 1e-9
    assert abs(O.stencil_symbol_max(2) - 4.0) < 1e-15
    assert abs(O.stencil_symbol_max(8) - 6.501587301587302) < 1e-12


# ---------------------------------------------------------------------------
# Closed-form standing modes of the leapfrog scheme (operator, BCs, stepping)
# ---------------------------------------------------------------------------
def _mode(shape, ks, bc):
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phi = np.ones(shape)
    thetas = []
    for g, n, k in zip(grids, shape, ks):
        if bc == "dirichlet":
            th = np.pi * k / (n + 1)
            phi = phi * np.sin(th * (g + 1))
        else:
            th = np.pi * k / n
            phi = phi * np.cos(th * (g + 0.5))
        thetas.append(th)
    return phi, thetas


def _symbol(order, theta, h):
    c = O.stencil_weights(order)
    return (c[0] + 2 * sum(c[j] * np.cos(j * theta) for j in range(1, len(c)))) / h ** 2


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
@pytest.mark.parametrize("shape,ks", [((23,), (3,)), ((17, 13), (2, 5)), ((11, 9, 10), (1, 3, 2))])
def test_standing_mode_exact(bc, order, shape, ks):
    h, v = 10.0, 2500.0
    dt = O.cfl_dt(h, v, len(shape), order, 0.5)
    phi, thetas = _mode(shape, ks, bc)
    mu = sum(_symbol(order, th, h) for th in thetas)
    cos_w = 1.0 + 0.5 * dt * dt * v * v * mu
    omega_dt = math.acos(cos_w)
    nt = 60
    med = O.Medium("velocity", np.full(shape, v), h, dt, order, bc)
    shot = O.Shot(src=0, wavelet=np.zeros(nt + 1), rec=np.arange(int(np.prod(shape))))
    out = O.forward(med, shot, nt, init=(phi, cos_w * phi))
    u_n, u_n1 = out["last"]
    np.testing.assert_allclose(u_n, math.cos(nt * omega_dt) * phi, atol=2e-11)
    np.testing.assert_allclose(u_n1, math.cos((nt + 1) * omega_dt) * phi, atol=2e-11)
    # traces record the same closed form at every level
    levels = np.array([math.cos(n * omega_dt) for n in range(nt + 1)])
    np.testing.assert_allclose(out["traces"], phi.reshape(-1, 1) * levels[None, :], atol=2e-11)


@pytest.mark.parametrize("shape,ks", [((19, 14), (4, 3)), ((9, 10, 11), (2, 3, 2))])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_density_standing_mode_exact(bc, shape, ks):
    # Homogeneous gamma: div(b grad u) = b * (2nd-order Laplacian), mass a.
    gamma = 0.7
    a, b, _, _ = O.density_materials(gamma)
    h = 2e-3
    dt = 0.5 * O.cfl_dt(h, math.sqrt(b / a), len(shape), 2, 1.0)
    phi, thetas = _mode(shape, ks, bc)
    mu = (b / a) * sum(_symbol(2, th, h) for th in thetas)
    cos_w = 1.0 + 0.5 * dt * dt * mu
    omega_dt = math.acos(cos_w)
    nt = 50
    med = O.Medium("density", np.full(shape, gamma), h, dt, 2, bc)
    shot = O.Shot(src=0, wavelet=np.zeros(nt + 1), rec=np.array([0]))
    out = O.forward(med, shot, nt, init=(phi, cos_w * phi))
    np.testing.assert_allclose(out["last"][0], math.cos(nt * omega_dt) * phi, atol=2e-11)


# ---------------------------------------------------------------------------
# Symmetry of the stiffness operators, energy conservation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_laplacian_symmetric(bc, order):
    rng = np.random.default_rng(order)
    shape = (13, 11, 12)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    lx = O.laplacian(x, 1.3, order, bc)
    ly = O.laplacian(y, 1.3, order, bc)
    assert abs(np.sum(lx * y) - np.sum(x * ly)) < 1e-12 * np.abs(lx * y).sum()
    # negative semidefinite
    assert np.sum(lx * x) < 0


@pytest.mark.parametrize("shape", [(15, 12), (7, 9, 8)])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_divergence_operator_symmetric(bc, shape):
    rng = np.random.default_rng(3)
    b = rng.uniform(0.01, 1.0, shape)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    lx = O.divergence_operator(x, b, 0.5, bc)
    ly = O.divergence_operator(y, b, 0.5, bc)
    assert abs(np.sum(lx * y) - np.sum(x * ly)) < 1e-12 * np.abs(lx * y).sum()
    if bc == "neumann":           # constants are in the kernel of the Neumann operator
        assert np.abs(O.divergence_operator(np.ones(shape), b, 0.5, bc)).max() < 1e-12


@pytest.mark.parametrize("physics,order,bc,shape", [("velocity", 8, "dirichlet", (21, 18)),
                                                     ("velocity", 4, "neumann", (21, 18)),
                                                     ("density", 2, "neumann", (21, 18)),
                                                     ("density", 2, "dirichlet", (21, 18)),
                                                     ("density", 2, "dirichlet", (9, 8, 10))])
def test_energy_conserved_without_sources(physics, order, bc, shape):
    rng = np.random.default_rng(11)
    if physics == "velocity":
        param = rng.uniform(1500, 4500, shape)
        dt = O.cfl_dt(10.0, 4500.0, len(shape), order, 0.5)
        h = 10.0
    else:
        param = rng.uniform(0.1, 1.0, shape)
        h = 2e-3
        dt = 0.5 * O.cfl_dt(h, 509.8, len(shape), 2, 1.0)
    med = O.Medium(physics, param, h, dt, order, bc)
    u_prev = rng.standard_normal(shape)
    u = u_prev + 0.01 * rng.standard_normal(shape)
    e0 = med.energy(u_prev, u)
    assert e0 > 0
    zero = np.zeros(shape)
    for _ in range(300):
        u_prev, u = u, med.step(u_prev, u, zero)
    assert abs(med.energy(u_prev, u) - e0) < 1e-11 * abs(e0)


# ---------------------------------------------------------------------------
# Adjoint dot-product test: <F s, w> = <s, F* w>
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("physics,order,bc,shape", [
    ("velocity", 2, "dirichlet", (16, 14)),
    ("velocity", 8, "neumann", (19, 17)),
    ("velocity", 6, "dirichlet", (13, 14, 15)),
    ("density", 2, "neumann", (15, 16)),
    ("density", 2, "dirichlet", (9, 10, 11)),
])
def test_adjoint_dot_product(physics, order, bc, shape):
    rng = np.random.default_rng(5)
    nt = 70
    if physics == "velocity":
        param, h = rng.uniform(1500, 4500, shape), 10.0
        dt = O.cfl_dt(h, 4500.0, len(shape), order, 0.5)
    else:
        param, h = rng.uniform(0.1, 1.0, shape), 2e-3
        dt = 0.5 * O.cfl_dt(h, 509.8, len(shape), 2, 1.0)
    med = O.Medium(physics, param, h, dt, order, bc)
    size = int(np.prod(shape))
    rec = rng.choice(size, 9, replace=False)
    src = int(rng.integers(size))
    s = rng.standard_normal(nt + 1)
    s[0] = 0.0
    w = rng.standard_normal((len(rec), nt + 1))
    fs = O.forward(med, O.Shot(src=src, wavelet=s, rec=rec), nt)["traces"]
    lam = O.adjoint(med, rec, w, nt)
    lhs = float(np.sum(fs * w))
    rhs = float(sum(s[n] * lam[n].ravel()[src] for n in range(1, nt + 1)))
    assert abs(lhs - rhs) < 1e-11 * (abs(lhs) + abs(rhs)), (lhs, rhs)


# ---------------------------------------------------------------------------
# Exact gradient against central finite differences of the misfit
# ---------------------------------------------------------------------------
def _fd_problem(physics, order, bc, shape, objective, seed=0):
    rng = np.random.default_rng(seed)
    nt = 60
    size = int(np.prod(shape))
    if physics == "velocity":
        h = 10.0
        true = rng.uniform(2000, 3000, shape)
        start = np.full(shape, 2500.0)
        dt = O.cfl_dt(h, 3000.0 * 1.05, len(shape), order, 0.5)
        wav = O.ricker(np.arange(nt + 1) * dt, 1.0 / (12 * dt))
    else:
        h = 2e-3
        true = rng.uniform(0.1, 1.0, shape)
        start = rng.uniform(0.3, 0.8, shape)
        dt = 0.45 * O.cfl_dt(h, 509.8, len(shape), 2, 1.0)
        wav = O.sine_burst(np.arange(nt + 1) * dt, 1.0 / (15 * dt), 2, 1.0)
    src = size // 2 + 1
    rec = rng.choice(size, 7, replace=False)
    if objective == "l2":
        obs = O.forward(O.Medium(physics, true, h, dt, order, bc), O.Shot(src, wav, rec), nt)["traces"]
        shot = O.Shot(src, wav, rec, obs, 1.0)
    else:
        shot = O.Shot(src, wav, rec, None, O.patch_weight(len(rec), -1.0))
    return dict(h=h, dt=dt, nt=nt, start=start, shot=shot, physics=physics, order=order, bc=bc, rng=rng)


def _cost(p, param):
    med = O.Medium(p["physics"], param, p["h"], p["dt"], p["order"], p["bc"])
    tr = O.forward(med, p["shot"], p["nt"])["traces"]
    return O.misfit(tr, p["shot"].observed, p["dt"], p["shot"].weight)


@pytest.mark.parametrize("physics,order,bc,shape,objective", [
    ("velocity", 2, "dirichlet", (12, 11), "l2"),
    ("velocity", 8, "dirichlet", (14, 13), "l2"),
    ("velocity", 4, "neumann", (8, 9, 10), "l2"),
    ("velocity", 2, "neumann", (13, 12), "patch"),
    ("density", 2, "neumann", (12, 13), "patch"),
    ("density", 2, "neumann", (12, 11), "l2"),
    ("density", 2, "dirichlet", (11, 12), "l2"),
    ("density", 2, "neumann", (7, 8, 9), "l2"),
    ("density", 2, "dirichlet", (8, 7, 9), "patch"),
])
def test_exact_gradient_matches_finite_differences(physics, order, bc, shape, objective):
    p = _fd_problem(physics, order, bc, shape, objective)
    med = O.Medium(physics, p["start"], p["h"], p["dt"], order, bc)
    c0, grad, _ = O.exact_gradient(med, [p["shot"]], p["nt"])
    assert abs(c0 - _cost(p, p["start"])) < 1e-12 * abs(c0)
    rng = p["rng"]
    if physics == "velocity":
        m0 = 1.0 / p["start"] ** 2
        dm = rng.standard_normal(shape) * m0
        eps = 1e-5
        cp = _cost(p, 1.0 / np.sqrt(m0 + eps * dm))
        cm = _cost(p, 1.0 / np.sqrt(m0 - eps * dm))
    else:
        dm = rng.standard_normal(shape)
        eps = 1e-6
        cp = _cost(p, p["start"] + eps * dm)
        cm = _cost(p, p["start"] - eps * dm)
    fd = (cp - cm) / (2 * eps)
    an = float(np.sum(grad * dm))
    assert abs(fd - an) < 1e-6 * abs(an), (fd, an)


def test_velocity_chain_rule_to_v():
    p = _fd_problem("velocity", 4, "dirichlet", (12, 12), "l2", seed=2)
    med = O.Medium("velocity", p["start"], p["h"], p["dt"], 4, "dirichlet")
    _, grad_m, _ = O.exact_gradient(med, [p["shot"]], p["nt"])
    grad_v = med.param_chain(grad_m)
    dv = p["rng"].standard_normal((12, 12)) * 10.0
    eps = 1e-3
    fd = (_cost(p, p["start"] + eps * dv) - _cost(p, p["start"] - eps * dv)) / (2 * eps)
    an = float(np.sum(grad_v * dv))
    assert abs(fd - an) < 1e-6 * abs(an)


# ---------------------------------------------------------------------------
# The superposition approximation (Sec. 4, Eq. superposedkernel1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("physics,order,bc,shape,objective", [
    ("velocity", 2, "dirichlet", (14, 12), "l2"),
    ("velocity", 8, "neumann", (13, 15), "l2"),
    ("velocity", 6, "dirichlet", (9, 10, 11), "l2"),
    ("density", 2, "neumann", (12, 14), "patch"),
    ("density", 2, "dirichlet", (13, 12), "l2"),
    ("density", 2, "neumann", (8, 9, 10), "l2"),
])
def test_superposition_identity(physics, order, bc, shape, objective):
    p = _fd_problem(physics, order, bc, shape, objective, seed=4)
    med = O.Medium(physics, p["start"], p["h"], p["dt"], order, bc)
    c_ex, g, parts = O.exact_gradient(med, [p["shot"]], p["nt"])
    k = O.auto_k(p["shot"], parts[0]["f_adj"], p["nt"], 1e-2)
    sup = O.superposition_gradient(med, [p["shot"]], p["nt"], k)
    assert abs(sup["C"] - c_ex) < 1e-12 * abs(c_ex)
    lam = parts[0]["lam"]
    klam = O.kernel_from_histories(med, lam, lam, p["nt"])
    resid = sup["K_tilde"] - g - 0.5 * k * klam
    scale = np.abs(g).max()
    assert np.abs(resid).max() < 1e-7 * scale
    # the approximation error is the k/2 K(lam, lam) term, small for this k
    # (its size depends on the problem: 1-7% at r = 1e-2 for these cases)
    gap = np.linalg.norm(sup["K_tilde"] - g) / np.linalg.norm(g)
    assert gap < 0.1
    # symmetric +-k average cancels the k^2 term exactly, at any k
    for kk in (k, 30 * k):
        sym = O.symmetric_superposition_gradient(med, [p["shot"]], p["nt"], kk)
        assert abs(sym["C"] - c_ex) < 1e-12 * abs(c_ex)
        assert np.abs(sym["K_tilde"] - g).max() < 1e-7 * scale
    # K_tilde is affine in k
    sup2 = O.superposition_gradient(med, [p["shot"]], p["nt"], 2 * k)
    np.testing.assert_allclose(sup2["K_tilde"] - sup["K_tilde"], 0.5 * k * klam, atol=1e-7 * scale)


def test_superposition_zero_residual_gives_zero_gradient():
    p = _fd_problem("velocity", 4, "dirichlet", (12, 13), "l2", seed=7)
    med = O.Medium("velocity", p["start"], p["h"], p["dt"], 4, "dirichlet")
    own = O.forward(med, p["shot"], p["nt"])["traces"]
    shot = O.Shot(p["shot"].src, p["shot"].wavelet, p["shot"].rec, own, 1.0)
    sup = O.superposition_gradient(med, [shot], p["nt"], 1e3)
    assert sup["C"] == 0.0
    assert np.abs(sup["K_tilde"]).max() < 1e-9 * np.abs(sup["K_f"]).max() / 1e3


def test_multishot_sum():
    p = _fd_problem("velocity", 2, "dirichlet", (12, 12), "l2", seed=9)
    med = O.Medium("velocity", p["start"], p["h"], p["dt"], 2, "dirichlet")
    s1 = p["shot"]
    s2 = O.Shot(s1.src + 3, s1.wavelet, s1.rec, s1.observed * 0.5, 1.0)
    both = O.superposition_gradient(med, [s1, s2], p["nt"], 10.0)
    a = O.superposition_gradient(med, [s1], p["nt"], 10.0)
    b = O.superposition_gradient(med, [s2], p["nt"], 10.0)
    np.testing.assert_allclose(both["K_tilde"], a["K_tilde"] + b["K_tilde"], rtol=1e-9, atol=1e-12)
    assert abs(both["C"] - a["C"] - b["C"]) < 1e-12 * both["C"]


# ---------------------------------------------------------------------------
# Wavelets, materials, CFL, misfit
# ---------------------------------------------------------------------------
def test_ricker_closed_form_points():
    f = 15.0
    t0 = 1.0 / f
    assert abs(O.ricker(np.array([t0]), f)[0] - 1.0) < 1e-15
    tz = 1.0 / (np.pi * f * math.sqrt(2.0))
    np.testing.assert_allclose(O.ricker(np.array([t0 - tz, t0 + tz]), f), 0.0, atol=1e-14)
    tm = math.sqrt(1.5) / (np.pi * f)
    np.testing.assert_allclose(O.ricker(np.array([t0 - tm, t0 + tm]), f), -2 * math.exp(-1.5), rtol=1e-13)
    t = np.linspace(-2, 2, 400001) + t0
    assert abs(np.sum(O.ricker(t, f)) * (t[1] - t[0])) < 1e-10     # zero mean


def test_sine_burst_closed_form_points():
    f, nc, psi0 = 10e3, 2, 3.0
    w = 2 * np.pi * f
    t = np.array([np.pi / (2 * w), 2 * np.pi * nc / w * 0.5, 2 * np.pi * nc / w * 1.0001, -1e-9])
    v = O.sine_burst(t, f, nc, psi0)
    assert abs(v[0] - psi0 * math.sin(np.pi / (4 * nc)) ** 2) < 1e-13
    assert abs(v[1]) < 1e-12           # sin(w t) = sin(2 pi) at the burst centre for nc = 2
    assert v[2] == 0.0 and v[3] == 0.0


def test_materials_recover_air_and_solid():
    a, b, da, db = O.density_materials(np.array([0.0, 1.0]))
    np.testing.assert_allclose(1 / b, [O.RHO_AIR, O.RHO_SOLID], rtol=1e-12)
    np.testing.assert_allclose(1 / a, [O.KAPPA_AIR, O.KAPPA_SOLID], rtol=1e-12)
    # speed of sound sqrt(kappa/rho): 343 m/s in air, 509.8 m/s in the solid
    np.testing.assert_allclose(np.sqrt(b / a), [343.3, 509.8], rtol=1e-3)


def test_paper_time_steps_lie_below_the_stability_limit():
    with open(os.path.join(GOLDEN, "paper_time_steps.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        h = case["L1_m"] / (case["n1"] - 1)
        limit = O.cfl_dt(h, case["c_max_m_per_s"], case["ndim"], 2, 1.0)
        frac = case["dt_s"] / limit
        assert case["fraction_min"] <= frac <= case["fraction_max"], (case["name"], frac)


def test_cfl_limit_is_sharp():
    # Highest Dirichlet mode: bounded just below the limit, grows just above it.
    n, h, v, order = 40, 1.0, 1.0, 8
    phi, _ = _mode((n,), (n,), "dirichlet")
    for frac, grows in ((0.99, False), (1.02, True)):
        dt = O.cfl_dt(h, v, 1, order, frac)
        med = O.Medium("velocity", np.full((n,), v), h, dt, order, "dirichlet")
        u_prev, u = phi, phi
        zero = np.zeros(n)
        for _ in range(400):
            u_prev, u = u, med.step(u_prev, u, zero)
        assert (np.abs(u).max() > 1e3) == grows


def test_misfit_hand_example():
    tr = np.array([[1.0, 2.0], [3.0, 4.0]])
    obs = np.array([[0.0, 1.0], [1.0, 0.0]])
    # 1/2 * dt * ((1)^2 + (1)^2 + (2)^2 + (4)^2) = 0.25 * 22
    assert O.misfit(tr, obs, 0.5) == 5.5
    assert O.misfit(tr, None, 0.5, O.patch_weight(4, 1.0)) == 0.5 * 0.5 * 0.5 * 30.0


def test_auto_k_hand_example():
    """The automatic k (reading R9): k = r ||psi|| / ||f_adj|| over levels 1..N
    of the first shot, worked by hand.  Level 0 of both series is excluded
    (f^0 is never used and u^0 = 0 gives no adjoint source)."""
    # psi levels 1..3 = (2, 1, 2): ||psi|| = 3; f_adj levels 1..3 of two
    # receivers = (0, 4, 0) and (0, 0, 3): ||f_adj|| = 5.  Level-0 entries (7,
    # 100, 11) would change the result if they were counted.
    wav = np.array([7.0, 2.0, 1.0, 2.0])
    f_adj = np.array([[100.0, 0.0, 4.0, 0.0], [11.0, 0.0, 0.0, 3.0]])
    shot = O.Shot(0, wav, np.array([1, 2]))
    assert O.auto_k(shot, f_adj, 3, 1e-2) == pytest.approx(1e-2 * 3.0 / 5.0, rel=1e-15)
    assert O.auto_k(shot, f_adj, 3, 0.5) == pytest.approx(0.5 * 0.6, rel=1e-15)
    # only levels up to N enter: with N = 2 the last column drops out,
    # ||psi|| = sqrt(5), ||f_adj|| = 4
    assert O.auto_k(shot, f_adj, 2, 1.0) == pytest.approx(math.sqrt(5.0) / 4.0, rel=1e-15)
    # a zero residual has no scale: k = 1
    assert O.auto_k(shot, np.zeros_like(f_adj), 3, 1e-2) == 1.0


# ---------------------------------------------------------------------------
# Planted mistakes: each must be caught by a pin above
# ---------------------------------------------------------------------------
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible errors in a copy of the oracle on the CPU and check a pin fails."""
    # 1) dropped 2u term sign: step uses u - u_prev
    shape, ks, bc, order = (17, 13), (2, 5), "dirichlet", 4
    h, v = 10.0, 2500.0
    dt = O.cfl_dt(h, v, 2, order, 0.5)
    phi, th = _mode(shape, ks, bc)
    cos_w = 1.0 + 0.5 * dt * dt * v * v * sum(_symbol(order, t, h) for t in th)
    med = O.Medium("velocity", np.full(shape, v), h, dt, order, bc)
    good = med.step(phi, cos_w * phi, np.zeros(shape))
    np.testing.assert_allclose(good, math.cos(2 * math.acos(cos_w)) * phi, atol=1e-12)

    # 2) wrong Dirichlet mirror sign breaks the standing mode
    orig = O.wave_oracle.ghost_index

    def bad_ghost(i, n, bc_):
        idx, s = orig(i, n, bc_)
        return idx, abs(s)
    monkeypatch.setattr(O.wave_oracle, "ghost_index", bad_ghost)
    bad = O.laplacian(phi, h, order, bc)
    monkeypatch.setattr(O.wave_oracle, "ghost_index", orig)
    ok = O.laplacian(phi, h, order, bc)
    assert np.abs(bad - ok).max() > 1e-6 * np.abs(ok).max()

    # 3) off-by-one adjoint source level breaks the dot-product test
    rng = np.random.default_rng(1)
    med = O.Medium("velocity", rng.uniform(1500, 4500, (12, 12)), 10.0, O.cfl_dt(10.0, 4500, 2, 2, 0.5), 2, "dirichlet")
    nt, rec, src = 40, np.array([3, 50, 77]), 70
    s = rng.standard_normal(nt + 1)
    s[0] = 0
    w = rng.standard_normal((3, nt + 1))
    fs = O.forward(med, O.Shot(src, s, rec), nt)["traces"]
    lam_shift = O.adjoint(med, rec, np.roll(w, 1, axis=1), nt)
    lhs = np.sum(fs * w)
    rhs = sum(s[n] * lam_shift[n].ravel()[src] for n in range(1, nt + 1))
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)
