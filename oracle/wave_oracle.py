"""FP64 CPU oracle for the memory-efficient (superposition) adjoint method.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
statement of what the GPU library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA path
and imports nothing from the package.

What it follows (arXiv 2509.15744, Herrmann, Buerchner, Kollmannsberger):

* Sec. 2.2 / 2.3: the scalar wave equation (Eq. scalarwaveequation, here in its
  squared-slowness form m u_tt - lap u = f) and the variable-density acoustic
  equation (Eq. wavetopopt) with the linear material interpolation of Sec. 2.3;
  point source with the Kronecker delta (Eq. source1), sine burst (Eq. source2);
  L2 trace misfit (Eq. cost1) and patch energy (Eq. cost2); adjoint sources
  (Eq. adjointSource1, Eq. adjointSource2); Frechet kernels (Eq. kernel1,
  Eq. kernel2).
* Sec. 3.1: leapfrog in time, central differences in space (Eq. FDstencil1,
  Eq. FDstencil2) with harmonic-mean faces and ghost cells whose material equals
  the boundary material.  Orders 4/6/8 use the textbook central weights.
* Sec. 4: superposed field u^s = u + k u_adj (Eq. superposedPDE,
  Eq. superposedforce), the kernel identity (Eq. superposedkernel1), the mixed
  kernel approximation (Eq. superposedkernel) and Algorithm 1.

Readings where the paper is silent or ambiguous (each is also listed in the
design notes of the repository):

R1  Velocity form: the mass is m = 1/v^2 and the stiffness the order-p
    Laplacian, u^{n+1} = 2u^n - u^{n-1} + (dt^2/m)(L u^n + f^n).
R2  Boundaries: Dirichlet is the odd mirror about the virtual wall nodes -1
    and n; Neumann (Eq. BC) is the even mirror about the half cell.  Both keep
    the discrete operator symmetric.
R3  Harmonic-mean faces: b_f = 2 b_i b_j / (b_i + b_j) with b = 1/rho, as in
    Eq. FDstencil2 and App. A.  Ghost material = boundary material (Sec. 3.1).
R4  Source: Kronecker point source, f_i^n = psi(n dt) at the source cell, no
    1/h^d factor.  Ricker wavelet with t0 = 1/f; sine burst with psi0 = 1.
R5  Time quadrature: rectangle rule, C = 1/2 w dt sum_{n=0}^{N} sum_r e_r^n^2,
    with traces at levels 0..N.  Patch energy is the same form with d = 0 and
    w = +-2/n_s (n_s = number of patch cells, the Kronecker-normalised area).
R6  Adjoint source in the paper's scaling: f_adj^n = -w e^n at the receivers
    (Eq. adjointSource1), so u^s = u + k u_adj exactly as in Sec. 4.
R7  End conditions: Algorithm 1 starts the superposed pass from levels N and
    N-1, which drops the adjoint source of level N.  Here the forward takes one
    extra (unrecorded) step to level N+1 and the superposed pass starts from
    (u^{N+1}, u^N) with j = N..1; this is the exact discrete adjoint.
R8  Discrete kernel: K(a, b) = -(da/dgamma)/dt sum_n Da Db over half levels
    (the discrete -int a' a_t b_t dt) plus, for the density form,
    (dt/h^2) sum_n sum_faces (d b_f / d gamma_i) D_f a D_f b (the discrete
    +int b' grad a . grad b dt of Eq. kernel2).  The half level N+1/2 and the
    level N are shared exactly by u and u^s and are left out of both sums.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
from typing import Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Materials of the acoustic (TATO) model, Sec. 2.3
# ---------------------------------------------------------------------------
RHO_AIR = 1.204          # kg/m^3
KAPPA_AIR = 1.419e5      # N/m^2
RHO_SOLID = 2643.0       # kg/m^3
KAPPA_SOLID = 6.87e8     # N/m^2 (the paper's reduced value, Sec. 2.3 footnote)


def density_materials(gamma: np.ndarray):
    """Linear interpolation of rho^-1 and kappa^-1 in gamma (Sec. 2.3).

    Returns (a, b, da, db): a = kappa^-1(gamma) is the mass coefficient,
    b = rho^-1(gamma) the stiffness coefficient, da and db their (constant)
    derivatives with respect to gamma.
    """
    gamma = np.asarray(gamma, dtype=np.float64)
    db = 1.0 / RHO_SOLID - 1.0 / RHO_AIR
    da = 1.0 / KAPPA_SOLID - 1.0 / KAPPA_AIR
    b = 1.0 / RHO_AIR + gamma * db
    a = 1.0 / KAPPA_AIR + gamma * da
    return a, b, da, db


# ---------------------------------------------------------------------------
# Central second-derivative weights (Sec. 3.1 is 2nd order; orders 4-8 are the
# textbook central weights c_0..c_r of d^2/dx^2, before the 1/h^2 factor).
# ---------------------------------------------------------------------------
SECOND_DERIVATIVE_WEIGHTS = {
    2: (Fraction(-2), Fraction(1)),
    4: (Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)),
    6: (Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)),
    8: (Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315),
        Fraction(-1, 560)),
}


def stencil_weights(order: int) -> np.ndarray:
    """c_0..c_r for the given even order as float64."""
    return np.array([float(c) for c in SECOND_DERIVATIVE_WEIGHTS[order]])


def stencil_symbol_max(order: int) -> float:
    """S = |c_0 + 2 sum_j (-1)^j c_j|: the largest |symbol| (at theta = pi)."""
    c = SECOND_DERIVATIVE_WEIGHTS[order]
    s = c[0] + 2 * sum(((-1) ** j) * c[j] for j in range(1, len(c)))
    return float(abs(s))


def cfl_dt(h: float, vmax: float, ndim: int, order: int,
           fraction: float = 0.5) -> float:
    """Time step at `fraction` of the leapfrog stability limit.

    Leapfrog is stable while dt^2 * max|eig(L)| * v^2 <= 4; for the order-p
    Laplacian max|eig| = ndim * S / h^2, so dt_max = 2 h / (v sqrt(ndim S)).
    """
    return fraction * 2.0 * h / (vmax * np.sqrt(ndim * stencil_symbol_max(order)))


# ---------------------------------------------------------------------------
# Ghost cells (Sec. 3.1 and reading R2)
# ---------------------------------------------------------------------------
def ghost_index(i: int, n: int, bc: str):
    """Map a possibly-outside index i of an axis of length n to (index, sign).

    Inside: (i, +1).  Neumann: even mirror about the half cell,
    u_{-1-j} = u_j.  Dirichlet: odd mirror about the virtual nodes -1 and n,
    u_{-1} = 0 and u_{-1-j} = -u_{j-1}.  A zero value is returned as (0, 0).
    """
    if 0 <= i < n:
        return i, 1.0
    if bc == "neumann":
        return (-1 - i, 1.0) if i < 0 else (2 * n - 1 - i, 1.0)
    if bc == "dirichlet":
        if i == -1 or i == n:
            return 0, 0.0
        return (-2 - i, -1.0) if i < 0 else (2 * n - i, -1.0)
    raise ValueError(bc)


def pad_axis(u: np.ndarray, axis: int, r: int, bc: str) -> np.ndarray:
    """Extend u by r ghost cells on both ends of one axis."""
    n = u.shape[axis]
    idx, sgn = zip(*(ghost_index(i, n, bc) for i in range(-r, n + r)))
    out = np.take(u, np.array(idx), axis=axis)
    shape = [1] * u.ndim
    shape[axis] = n + 2 * r
    return out * np.array(sgn).reshape(shape)


def pad_material_axis(b: np.ndarray, axis: int) -> np.ndarray:
    """One ghost cell per side whose material equals the boundary material."""
    n = b.shape[axis]
    idx = np.array([0] + list(range(n)) + [n - 1])
    return np.take(b, idx, axis=axis)


# ---------------------------------------------------------------------------
# Stiffness operators
# ---------------------------------------------------------------------------
def laplacian(u: np.ndarray, h: float, order: int, bc: str) -> np.ndarray:
    """Order-p central Laplacian, sum over axes of (1/h^2) sum_j c_j (u_{+j} + u_{-j})."""
    c = stencil_weights(order)
    r = len(c) - 1
    out = np.zeros_like(u, dtype=np.float64)
    for ax in range(u.ndim):
        n = u.shape[ax]
        p = pad_axis(u, ax, r, bc)
        acc = c[0] * u
        for j in range(1, r + 1):
            plus = np.take(p, np.arange(r + j, r + j + n), axis=ax)
            minus = np.take(p, np.arange(r - j, r - j + n), axis=ax)
            acc = acc + c[j] * (plus + minus)
        out += acc
    return out / (h * h)


def face_coefficients(b: np.ndarray, axis: int) -> np.ndarray:
    """Harmonic-mean faces b_f = 2 b_i b_j / (b_i + b_j) along one axis.

    Returns n+1 faces: face k sits between cells k-1 and k, faces 0 and n
    join a cell to its ghost (ghost material = boundary material, Sec. 3.1).
    """
    p = pad_material_axis(b, axis)
    n = b.shape[axis]
    left = np.take(p, np.arange(0, n + 1), axis=axis)
    right = np.take(p, np.arange(1, n + 2), axis=axis)
    return 2.0 * left * right / (left + right)


def divergence_operator(u: np.ndarray, b: np.ndarray, h: float, bc: str) -> np.ndarray:
    """Second-order div(b grad u) of Eq. FDstencil2, summed over axes.

    (1/h^2) [b_{i+1/2} (u_{i+1} - u_i) - b_{i-1/2} (u_i - u_{i-1})] per axis.
    """
    out = np.zeros_like(u, dtype=np.float64)
    for ax in range(u.ndim):
        n = u.shape[ax]
        p = pad_axis(u, ax, 1, bc)                     # n + 2 values
        bf = face_coefficients(b, ax)                  # n + 1 faces
        grad = np.diff(p, axis=ax)                     # n + 1 face differences
        flux = bf * grad
        out += np.take(flux, np.arange(1, n + 1), axis=ax) - np.take(flux, np.arange(0, n), axis=ax)
    return out / (h * h)


# ---------------------------------------------------------------------------
# The medium: mass a_i and stiffness L, and the leapfrog step
# ---------------------------------------------------------------------------
@dataclass
class Medium:
    """A discretised medium on a uniform grid (x fastest, C order)."""
    physics: str            # "velocity" (param = v [m/s]) or "density" (param = gamma)
    param: np.ndarray
    h: float
    dt: float
    order: int = 2
    bc: str = "dirichlet"

    def __post_init__(self):
        self.param = np.asarray(self.param, dtype=np.float64)
        if self.physics == "velocity":
            self.a = 1.0 / self.param ** 2         # squared slowness m (reading R1)
            self.b = None
            self.da = 1.0                          # d a / d m: the gradient is w.r.t. m
            self.db = 0.0
        elif self.physics == "density":
            if self.order != 2:
                raise ValueError("the density form is second order (Eq. FDstencil2)")
            self.a, self.b, self.da, self.db = density_materials(self.param)
        else:
            raise ValueError(self.physics)
        r = self.order // 2
        for n in self.param.shape:
            if n < 2 * r + 1:
                raise ValueError("each axis needs at least order+1 cells")

    @property
    def shape(self):
        return self.param.shape

    def stiffness(self, u: np.ndarray) -> np.ndarray:
        if self.physics == "velocity":
            return laplacian(u, self.h, self.order, self.bc)
        return divergence_operator(u, self.b, self.h, self.bc)

    def step(self, u_prev: np.ndarray, u: np.ndarray, f: np.ndarray) -> np.ndarray:
        """One leapfrog step (Eq. FDstencil1/2): 2u - u_prev + dt^2/a (L u + f)."""
        return 2.0 * u - u_prev + (self.dt ** 2 / self.a) * (self.stiffness(u) + f)

    def energy(self, u_prev: np.ndarray, u: np.ndarray) -> float:
        """Discrete energy of the leapfrog scheme at the half level between the
        two given levels: 1/2 sum a (Du/dt)^2 - 1/2 u^T L u_prev.  Constant in
        time without sources when L is symmetric."""
        du = (u - u_prev) / self.dt
        return 0.5 * float(np.sum(self.a * du * du)) - 0.5 * float(np.sum(u * self.stiffness(u_prev)))

    # -- discrete Frechet kernel, reading R8 ---------------------------------
    def kernel_half_level(self, da_: np.ndarray, db_: np.ndarray) -> np.ndarray:
        """Mass part at one half level: -(d a/d gamma)/dt * Da * Db (Eq. kernel1/2)."""
        return -(self.da / self.dt) * da_ * db_

    def kernel_level(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """Stiffness part at one integer level (density form only):
        (dt/h^2) sum over faces f of cell i of (d b_f/d gamma_i) D_f x D_f y,
        the discrete +int b' grad x . grad y dt of Eq. kernel2."""
        if self.physics == "velocity":
            return np.zeros(self.shape)
        out = np.zeros(self.shape)
        b = self.b
        for ax in range(x.ndim):
            n = x.shape[ax]
            px = pad_axis(x, ax, 1, self.bc)
            py = pad_axis(y, ax, 1, self.bc)
            pb = pad_material_axis(b, ax)
            for side in (+1, -1):
                # neighbour j = i + side along this axis
                xj = np.take(px, np.arange(1 + side, n + 1 + side), axis=ax)
                yj = np.take(py, np.arange(1 + side, n + 1 + side), axis=ax)
                bj = np.take(pb, np.arange(1 + side, n + 1 + side), axis=ax)
                # d b_f / d b_i for b_f = 2 b_i b_j/(b_i + b_j)
                dbf = 2.0 * bj * bj / (b + bj) ** 2
                # faces to ghost cells carry no flux under Neumann; under
                # Dirichlet the ghost material is the boundary material
                # itself, so d b_f/d gamma_i = db (b_f = b_i).
                term = self.db * dbf * (xj - x) * (yj - y)
                edge = [slice(None)] * x.ndim
                edge[ax] = 0 if side < 0 else n - 1
                if self.bc == "neumann":
                    term[tuple(edge)] = 0.0
                else:
                    xe = (xj - x)[tuple(edge)]
                    ye = (yj - y)[tuple(edge)]
                    term[tuple(edge)] = self.db * xe * ye
                out += term
        return (self.dt / self.h ** 2) * out

    def param_chain(self, grad_a: np.ndarray) -> np.ndarray:
        """dC/dv from dC/dm for the velocity form (m = 1/v^2)."""
        if self.physics != "velocity":
            return grad_a
        return grad_a * (-2.0 / self.param ** 3)


# ---------------------------------------------------------------------------
# Source time functions (Eq. source2 and the Ricker wavelet, reading R4)
# ---------------------------------------------------------------------------
def ricker(t: np.ndarray, f: float, t0: Optional[float] = None) -> np.ndarray:
    """(1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0, t0 = 1/f."""
    t0 = 1.0 / f if t0 is None else t0
    a = (np.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def sine_burst(t: np.ndarray, f: float, nc: int = 2, psi0: float = 1.0) -> np.ndarray:
    """psi0 sin(w t) sin^2(w t / (2 nc)) for 0 <= t <= 2 pi nc / w, else 0 (Eq. source2)."""
    t = np.asarray(t, dtype=np.float64)
    w = 2.0 * np.pi * f
    val = psi0 * np.sin(w * t) * np.sin(w * t / (2 * nc)) ** 2
    return np.where((t >= 0) & (t <= 2 * np.pi * nc / w), val, 0.0)


# ---------------------------------------------------------------------------
# Shots, objective, forward problem
# ---------------------------------------------------------------------------
@dataclass
class Shot:
    """One source with its receivers.

    src: flat (C-order) index of the source cell; wavelet: psi at t_n = n dt
    for n = 0..N (f^0 is never used); rec: flat receiver (or patch) indices;
    observed: [nrec, N+1] measured traces (None means zero, as for the patch
    energy); weight: w of reading R5 (1 for Eq. cost1, +-2/n_s for Eq. cost2).
    """
    src: int
    wavelet: np.ndarray
    rec: np.ndarray
    observed: Optional[np.ndarray] = None
    weight: float = 1.0

    def data(self, nt: int) -> np.ndarray:
        if self.observed is None:
            return np.zeros((len(self.rec), nt + 1))
        return np.asarray(self.observed, dtype=np.float64)


def patch_weight(n_patch: int, sign: float = 1.0) -> float:
    """w for the patch energy C = sign dt/n_s sum u^2 (Eq. cost2, reading R5)."""
    return 2.0 * sign / n_patch


def point_force(shape, cell: int, value: float) -> np.ndarray:
    """Kronecker point force (Eq. source1)."""
    f = np.zeros(int(np.prod(shape)))
    f[cell] = value
    return f.reshape(shape)


def forward(med: Medium, shot: Shot, nt: int, init=None, keep_history: bool = False):
    """Leapfrog forward problem, levels 0..N recorded, one extra step to N+1.

    init = (u^0, u^1) or None for the homogeneous initial conditions (Eq. IC).
    Returns dict(traces [nrec, N+1], last=(u^N, u^{N+1}), history=[u^0..u^{N+1}]).
    """
    shape = med.shape
    u_prev = np.zeros(shape) if init is None else np.asarray(init[0], np.float64).copy()
    u = np.zeros(shape) if init is None else np.asarray(init[1], np.float64).copy()
    rec = np.asarray(shot.rec)
    traces = np.zeros((len(rec), nt + 1))
    traces[:, 0] = u_prev.ravel()[rec]
    traces[:, 1] = u.ravel()[rec]
    history = [u_prev.copy(), u.copy()] if keep_history else None
    for n in range(1, nt + 1):
        u_next = med.step(u_prev, u, point_force(shape, shot.src, shot.wavelet[n]))
        if n + 1 <= nt:
            traces[:, n + 1] = u_next.ravel()[rec]
        if keep_history:
            history.append(u_next.copy())
        u_prev, u = u, u_next
    return dict(traces=traces, last=(u_prev, u), history=history)


def misfit(traces: np.ndarray, observed: Optional[np.ndarray], dt: float, weight: float = 1.0) -> float:
    """C = 1/2 w dt sum_n sum_r (u_r^n - d_r^n)^2 (Eq. cost1, rectangle rule, R5)."""
    d = 0.0 if observed is None else np.asarray(observed, np.float64)
    e = np.asarray(traces, np.float64) - d
    return 0.5 * weight * dt * float(np.sum(e * e))


def adjoint_source(traces: np.ndarray, shot: Shot, nt: int) -> np.ndarray:
    """f_adj^n_r = -w (u_r^n - d_r^n) (Eq. adjointSource1 / 2, reading R6)."""
    return -shot.weight * (traces - shot.data(nt))


def adjoint(med: Medium, rec: np.ndarray, f_adj: np.ndarray, nt: int, keep_history: bool = True):
    """Adjoint recursion backward in time with the end conditions Eq. ICadjoint.

    lam^{N+1} = lam^N = 0, lam^{j-1} = 2 lam^j - lam^{j+1} + dt^2/a (L lam^j + f_adj^j)
    for j = N..1, the adjoint injected at the receiver cells.
    Returns the list [lam^0 .. lam^{N+1}].
    """
    shape = med.shape
    size = int(np.prod(shape))
    lam_next = np.zeros(shape)   # lam^{j+1}
    lam = np.zeros(shape)        # lam^j
    levels = [None] * (nt + 2)
    levels[nt + 1] = lam_next.copy()
    levels[nt] = lam.copy()
    for j in range(nt, 0, -1):
        g = np.zeros(size)
        np.add.at(g, np.asarray(rec), f_adj[:, j])
        lam_prev = med.step(lam_next, lam, g.reshape(shape))
        levels[j - 1] = lam_prev
        lam_next, lam = lam, lam_prev
    return levels


def kernel_from_histories(med: Medium, x_hist: Sequence[np.ndarray], y_hist: Sequence[np.ndarray], nt: int) -> np.ndarray:
    """Discrete bilinear kernel K(x, y) of reading R8 over stored histories.

    Half levels n + 1/2 for n = 0..N-1 and integer levels n = 1..N-1.
    """
    out = np.zeros(med.shape)
    for n in range(0, nt):
        out += med.kernel_half_level(x_hist[n + 1] - x_hist[n], y_hist[n + 1] - y_hist[n])
    if med.physics == "density":
        for n in range(1, nt):
            out += med.kernel_level(x_hist[n], y_hist[n])
    return out


def exact_gradient(med: Medium, shots: Sequence[Shot], nt: int):
    """Standard (stored-history) adjoint gradient dC/dgamma = K(u_adj, u)
    (Eq. sensitivitygamma, Eq. gradientgamma), summed over shots.

    Returns (C, grad, per-shot dict with 'u' and 'lam' histories).
    """
    total_c = 0.0
    grad = np.zeros(med.shape)
    parts = []
    for shot in shots:
        fw = forward(med, shot, nt, keep_history=True)
        total_c += misfit(fw["traces"], shot.observed, med.dt, shot.weight)
        f_adj = adjoint_source(fw["traces"], shot, nt)
        lam = adjoint(med, shot.rec, f_adj, nt)
        grad += kernel_from_histories(med, lam, fw["history"], nt)
        parts.append(dict(u=fw["history"], lam=lam, traces=fw["traces"], f_adj=f_adj))
    return total_c, grad, parts


def auto_k(shot: Shot, f_adj: np.ndarray, nt: int, ratio: float = 1e-2) -> float:
    """k = ratio * ||psi|| / ||f_adj|| over levels 1..N (a stand-in for the
    calibration procedure of Sec. 4.1, which starts from a large k)."""
    psi = np.asarray(shot.wavelet[1:nt + 1], np.float64)
    g = np.asarray(f_adj[:, 1:nt + 1], np.float64)
    gn = float(np.sqrt(np.sum(g * g)))
    if gn == 0.0:
        return 1.0
    return ratio * float(np.sqrt(np.sum(psi * psi))) / gn


def superposition_gradient(med: Medium, shots: Sequence[Shot], nt: int, k: float):
    """Algorithm 1 (Sec. 4) with the end-condition reading R7, summed over shots.

    Forward loop: propagate, form the adjoint source, increment the cost and
    subtract the kernel K(u, u) of the new half level (and of the level n
    for the density form).  Then scale the adjoint force by k, start the
    superposed field from the forward's last two levels, and run backward in
    time adding K(u^s, u^s).  The result is K_tilde = (K(u^s,u^s) - K(u,u)) / (2k)
    (Eq. superposedkernel).

    Returns dict(C, K_tilde, K_f, K_s).
    """
    shape = med.shape
    total_c = 0.0
    k_f = np.zeros(shape)
    k_s = np.zeros(shape)
    for shot in shots:
        rec = np.asarray(shot.rec)
        d = shot.data(nt)
        size = int(np.prod(shape))
        # -- forward (Algorithm 1, forward loop) --------------------------
        u_prev = np.zeros(shape)
        u = np.zeros(shape)
        f_adj = np.zeros((len(rec), nt + 1))
        for level in (0, 1):
            e = (u.ravel()[rec] if level else u_prev.ravel()[rec]) - d[:, level]
            f_adj[:, level] = -shot.weight * e
            total_c += 0.5 * shot.weight * med.dt * float(np.sum(e * e))
        for n in range(1, nt + 1):
            u_next = med.step(u_prev, u, point_force(shape, shot.src, shot.wavelet[n]))
            if n + 1 <= nt:                                   # recorded levels only
                e = u_next.ravel()[rec] - d[:, n + 1]
                f_adj[:, n + 1] = -shot.weight * e            # computeAdjointSource
                total_c += 0.5 * shot.weight * med.dt * float(np.sum(e * e))  # incrementCost
            if n <= nt - 1:                                   # incrementKernel(u, u)
                k_f += med.kernel_half_level(u_next - u, u_next - u)
                k_f += med.kernel_level(u, u)
            u_prev, u = u, u_next
        # -- superposed pass (Algorithm 1, backward loop) -------------------
        scaled = k * f_adj                                    # scale adjoint force
        us_next, us = u, u_prev                               # u^{s,N+1}, u^{s,N}
        for j in range(nt, 0, -1):
            g = np.zeros(size)
            g[shot.src] += shot.wavelet[j]
            np.add.at(g, rec, scaled[:, j])
            us_prev = med.step(us_next, us, g.reshape(shape))  # u^{s,j-1}
            k_s += med.kernel_half_level(us - us_prev, us - us_prev)
            if j <= nt - 1:
                k_s += med.kernel_level(us, us)
            us_next, us = us, us_prev
    return dict(C=total_c, K_tilde=(k_s - k_f) / (2.0 * k), K_f=k_f, K_s=k_s)


def symmetric_superposition_gradient(med: Medium, shots: Sequence[Shot], nt: int, k: float):
    """Mean of the superposition result at +k and -k.

    K_tilde(k) = g + (k/2) K(u_adj, u_adj) (Eq. superposedkernel1 applied to
    the discrete bilinear kernel) is affine in k, so the mean over +-k drops
    the k^2 term and equals the exact gradient g; the forward kernel K(u, u)
    cancels as well, leaving (K(u^+,u^+) - K(u^-,u^-)) / 4k with
    u^+- = u +- k u_adj.

    Returns dict(C, K_tilde).
    """
    plus = superposition_gradient(med, shots, nt, k)
    minus = superposition_gradient(med, shots, nt, -k)
    return dict(C=plus["C"], K_tilde=0.5 * (plus["K_tilde"] + minus["K_tilde"]))
