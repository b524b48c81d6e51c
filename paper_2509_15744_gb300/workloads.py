"""Seeded synthetic inputs for the five benchmark workloads.

This module only builds inputs: model grids, source and receiver positions,
record lengths and the wavelet parameters.  It holds none of the method's
arithmetic (no stencil, time step rule, wavelet formula, misfit or kernel), so
both the FP64 oracle and the GPU library can consume what it returns.

The paper's own data (a CT-scanned cylinder, an acoustic black hole design)
are not available; these fields stand in for them with the structure of those
experiments: point sources on or near a surface, receiver lines or grids on
the surface, velocity contrast 1:1.5 to 1:3, smooth or layered media, and the
paper's density interpolation for the topology-optimisation case.

Grids are C-ordered numpy arrays (slowest axis first): (ny, nx) in 2D and
(nz, ny, nx) in 3D.  Cell indices are flat C-order indices.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class WaveletSpec:
    kind: str                 # "ricker" or "sine_burst"
    freq: float               # Hz
    nc: int = 2               # cycles of the sine burst
    psi0: float = 1.0         # amplitude


@dataclass
class Workload:
    name: str
    shape: tuple              # C order, slowest first
    h: float                  # grid spacing [m]
    order: int                # spatial order 2/4/6/8
    bc: str                   # "dirichlet" or "neumann"
    physics: str              # "velocity" (v [m/s]) or "density" (gamma)
    true_param: Optional[np.ndarray]   # model that generates the observed data
    init_param: np.ndarray    # model at which the gradient is taken
    vmax: float               # largest wave speed, for the time step rule
    cfl_fraction: float       # fraction of the stability limit
    sources: List[int]        # flat source cell per shot
    receivers: List[np.ndarray]  # flat receiver (or patch) cells per shot
    nt: List[int]             # record length N_s per shot
    wavelet: WaveletSpec
    objective: str = "l2"     # "l2" (Eq. cost1) or "patch" (Eq. cost2)
    patch_sign: float = 1.0   # +1 suppress, -1 amplify (patch objective)
    notes: str = ""

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def ncells(self):
        return int(np.prod(self.shape))

    @property
    def nshots(self):
        return len(self.sources)


def flat_index(shape, *coords):
    return int(np.ravel_multi_index(tuple(int(c) for c in coords), shape))


def _gaussian_smooth_noise(rng, shape, sigma):
    from scipy.ndimage import gaussian_filter
    noise = rng.standard_normal(shape)
    return gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)


def _minmax(x, lo, hi):
    x = (x - x.min()) / (x.max() - x.min())
    return lo + (hi - lo) * x


# ---------------------------------------------------------------------------
# Workload 0: 2D 128^2 circular inclusion, 2nd order, Dirichlet, 400 steps
# ---------------------------------------------------------------------------
def workload0(n: int = 128, nt: int = 400) -> Workload:
    shape = (n, n)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    c = n // 2
    r = 15 * n // 128
    true = np.full(shape, 2000.0, np.float32)
    true[(yy - c) ** 2 + (xx - c) ** 2 <= r * r] = 3000.0
    init = np.full(shape, 2000.0, np.float32)
    rec = np.array([flat_index(shape, 0, x) for x in range(0, n, 2)], np.int64)
    return Workload(
        name=f"2d_{n}x{n}_o2_inclusion", shape=shape, h=10.0, order=2, bc="dirichlet",
        physics="velocity", true_param=true, init_param=init, vmax=3000.0, cfl_fraction=0.5,
        sources=[flat_index(shape, 0, c)], receivers=[rec], nt=[nt],
        wavelet=WaveletSpec("ricker", 15.0),
        notes="true: 2000 m/s + 3000 m/s disc of radius 15 cells; initial: 2000 m/s")


# ---------------------------------------------------------------------------
# Workload 1: 2D 2048^2 smooth random field, 8th order, 4000 steps
# ---------------------------------------------------------------------------
def smooth_random_velocity(rng, shape, sigma, lo=1500.0, hi=4500.0):
    return _minmax(_gaussian_smooth_noise(rng, shape, sigma), lo, hi)


def workload1(n: int = 2048, nt: int = 4000, seed: int = 1) -> Workload:
    rng = np.random.default_rng(seed)
    shape = (n, n)
    sig = 50.0 * n / 2048
    noise = rng.standard_normal(shape)
    from scipy.ndimage import gaussian_filter
    true = _minmax(gaussian_filter(noise, sig, mode="reflect", truncate=4.0), 1500.0, 4500.0)
    init = _minmax(gaussian_filter(true, 4 * sig, mode="reflect", truncate=4.0), 1500.0, 4500.0)
    rec = np.array([flat_index(shape, 0, x) for x in range(0, n, 4)], np.int64)
    return Workload(
        name=f"2d_{n}x{n}_o8_smooth", shape=shape, h=10.0, order=8, bc="dirichlet",
        physics="velocity", true_param=true.astype(np.float32), init_param=init.astype(np.float32),
        vmax=4500.0, cfl_fraction=0.5, sources=[flat_index(shape, 0, n // 2)], receivers=[rec],
        nt=[nt], wavelet=WaveletSpec("ricker", 15.0),
        notes="Gaussian-filtered N(0,1) noise (sigma 50 cells) mapped to [1500, 4500]; "
              "initial = the same field filtered with sigma 200 cells")


# ---------------------------------------------------------------------------
# Workload 2: 3D 512^3 layered, 8th order, 16 shots with uneven lengths
# ---------------------------------------------------------------------------
def layered_profile(rng, nz, nlayers=8, lo=1500.0, hi=4500.0):
    depths = np.sort(rng.integers(1, nz, size=nlayers - 1))
    prof = np.empty(nz, np.float64)
    bounds = [0] + list(depths) + [nz]
    for i in range(nlayers):
        prof[bounds[i]:bounds[i + 1]] = lo + (hi - lo) * i / (nlayers - 1)
    return prof


def workload2(n: int = 512, nshots: int = 16, nt_range=(1500, 2500), rec_step: int = 2,
              seed: int = 2, src_depth: int = 2, rec_depth: int = 1, shape=None) -> Workload:
    rng = np.random.default_rng(seed)
    shape = (n, n, n) if shape is None else tuple(shape)
    nz, ny, nx = shape
    prof = layered_profile(rng, nz)
    from scipy.ndimage import gaussian_filter1d
    # The layers depend on depth only, so the 3D Gaussian filter of the model
    # (sigma 20 cells, reflect padding) is this 1D filter along depth.
    sprof = gaussian_filter1d(prof, 20.0 * nz / 512, mode="reflect", truncate=4.0)
    true = np.broadcast_to(prof.astype(np.float32)[:, None, None], shape)
    init = np.broadcast_to(sprof.astype(np.float32)[:, None, None], shape)
    side = int(round(np.sqrt(nshots)))
    sy = np.linspace(ny / (2 * side), ny - ny / (2 * side), side).astype(int)
    sx = np.linspace(nx / (2 * side), nx - nx / (2 * side), side).astype(int)
    sources = [flat_index(shape, src_depth, y, x) for y in sy for x in sx][:nshots]
    ry, rx = np.meshgrid(np.arange(0, ny, rec_step), np.arange(0, nx, rec_step), indexing="ij")
    rec = (rec_depth * ny * nx + ry * nx + rx).ravel().astype(np.int64)
    nts = [int(v) for v in rng.integers(nt_range[0], nt_range[1] + 1, size=nshots)]
    return Workload(
        name=f"3d_{nz}x{ny}x{nx}_o8_layered_{nshots}shots", shape=shape, h=10.0, order=8,
        bc="dirichlet", physics="velocity", true_param=true, init_param=init, vmax=4500.0,
        cfl_fraction=0.5, sources=sources, receivers=[rec] * nshots, nt=nts,
        wavelet=WaveletSpec("ricker", 15.0),
        notes="8 layers at sorted uniform random depths, 1500->4500 m/s with depth; "
              "initial = Gaussian smoothing (sigma 20 cells) along depth; "
              "sources on a 4x4 grid at depth 2, receivers every 2nd cell at depth 1")


# ---------------------------------------------------------------------------
# Workload 3: 2D 4096^2 variable-density acoustic (topology optimisation)
# ---------------------------------------------------------------------------
def workload3(n: int = 4096, nt: int = 6000, seed: int = 3, sign: float = 1.0) -> Workload:
    rng = np.random.default_rng(seed)
    shape = (n, n)
    gamma = rng.uniform(0.1, 1.0, shape).astype(np.float32)
    # Source at the left edge middle, as in the paper's layout.  The target
    # patch Omega_s is centred vertically but not at the far edge: with the
    # linear interpolation of 1/rho and 1/kappa the sound speed is ~343 m/s
    # for every gamma < 1, so 6000 steps of dt = 0.5 CFL (8.3 ms) carry the
    # burst ~1430 cells; the patch spans x in [n/8, 3n/16), which it reaches
    # after ~3 ms.
    y0, y1 = (3 * n) // 8, (5 * n) // 8
    x0, x1 = n // 8, n // 8 + max(1, n // 16)
    py, px = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    patch = (py * n + px).ravel().astype(np.int64)
    return Workload(
        name=f"2d_{n}x{n}_density_patch", shape=shape, h=2e-3, order=2, bc="neumann",
        physics="density", true_param=None, init_param=gamma, vmax=509.8366, cfl_fraction=0.5,
        sources=[flat_index(shape, n // 2, 2)], receivers=[patch], nt=[nt],
        wavelet=WaveletSpec("sine_burst", 10e3, 2, 1.0), objective="patch", patch_sign=sign,
        notes="gamma ~ U[0.1, 1] i.i.d.; sine burst 10 kHz, 2 cycles at the left edge middle; "
              "patch energy over x in [n/8, 3n/16), y in [3n/8, 5n/8)")


# ---------------------------------------------------------------------------
# Workload 4: 3D 1024^3 / 1536^3 smooth random velocity, 4 shots, 3000 steps
# ---------------------------------------------------------------------------
def smooth_field_3d(rng, shape, corr_cells, lo=1500.0, hi=4500.0, nmodes=48):
    """Smooth random field from a sum of random low-wavenumber plane cosines.

    Each mode is separable, so the field is one float32 matrix product
    [nz, nmodes] x [nmodes, ny*nx] and a 1e9-cell grid is cheap to build; the
    correlation length is about corr_cells.
    """
    nz, ny, nx = shape
    z = np.arange(nz, dtype=np.float32)
    y = np.arange(ny, dtype=np.float32)
    x = np.arange(nx, dtype=np.float32)
    zc = np.empty((nz, nmodes), np.float32)
    yx = np.empty((nmodes, ny * nx), np.float32)
    for m in range(nmodes):
        kz, ky, kx = rng.normal(0.0, 1.0 / corr_cells, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        amp = rng.normal()
        zc[:, m] = amp * np.cos(kz * z + ph[0])
        yx[m] = (np.cos(ky * y + ph[1])[:, None] * np.cos(kx * x + ph[2])[None, :]).ravel()
    out = (zc @ yx).reshape(shape)
    lo_v, hi_v = float(out.min()), float(out.max())
    out -= lo_v
    out *= (hi - lo) / (hi_v - lo_v)
    out += lo
    return out


def workload4(n: int = 1024, nshots: int = 4, nt: int = 3000, seed: int = 4) -> Workload:
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    true = smooth_field_3d(rng, shape, 50.0)
    init = smooth_field_3d(np.random.default_rng(seed + 100), shape, 200.0)
    side = 2
    s = [n // 3, 2 * n // 3]
    sources = [flat_index(shape, 2, y, x) for y in s for x in s][:nshots]
    step = max(1, n // 256)
    ry, rx = np.meshgrid(np.arange(0, n, step)[:256], np.arange(0, n, step)[:256], indexing="ij")
    rec = (1 * n * n + ry * n + rx).ravel().astype(np.int64)
    return Workload(
        name=f"3d_{n}^3_o8_smooth_{nshots}shots", shape=shape, h=10.0, order=8, bc="dirichlet",
        physics="velocity", true_param=true, init_param=init, vmax=4500.0, cfl_fraction=0.5,
        sources=sources, receivers=[rec] * nshots, nt=[nt] * nshots,
        wavelet=WaveletSpec("ricker", 15.0),
        notes="sum of 48 random plane cosines (correlation ~50 cells) mapped to [1500, 4500]")


def refined(w: Workload, factor: int = 2) -> Workload:
    """The same experiment on a grid `factor` times finer in every axis with
    `factor` times more, shorter steps, for observed data free of the
    'inverse crime' (the paper generates its data on a 2x grid with 2x steps).

    Grid nodes keep their positions (coarse node i is fine node factor*i);
    the true model is repeated into the new nodes; sources and receivers move
    to the matching fine nodes.  A Kronecker source of amplitude psi at one
    cell is a point source of strength psi h^d, so the fine grid injects
    psi * factor^d.  The wavelet is the same function of time, sampled at the
    fine step; level factor*n of the fine run is level n of the coarse axis
    (`coarse_samples`)."""
    f = int(factor)
    if f < 1:
        raise ValueError("factor must be >= 1")
    shape = tuple(n * f for n in w.shape)

    def up(a):
        if a is None:
            return None
        out = np.asarray(a)
        for ax in range(out.ndim):
            out = np.repeat(out, f, axis=ax)
        return np.ascontiguousarray(out)

    def move(cells):
        coords = np.unravel_index(np.asarray(cells, dtype=np.int64), w.shape)
        return np.ravel_multi_index(tuple(np.asarray(c) * f for c in coords), shape).astype(np.int64)

    wav = WaveletSpec(w.wavelet.kind, w.wavelet.freq, w.wavelet.nc, w.wavelet.psi0 * f ** len(w.shape))
    return Workload(
        name=f"{w.name}_refined{f}", shape=shape, h=w.h / f, order=w.order, bc=w.bc, physics=w.physics,
        true_param=up(w.true_param), init_param=up(w.init_param), vmax=w.vmax, cfl_fraction=w.cfl_fraction,
        sources=[int(move([s])[0]) for s in w.sources], receivers=[move(r) for r in w.receivers],
        nt=[n * f for n in w.nt], wavelet=wav, objective=w.objective, patch_sign=w.patch_sign,
        notes=f"{factor}x refinement of {w.name}")


def coarse_samples(traces: np.ndarray, factor: int = 2) -> np.ndarray:
    """Traces [nrec, factor*N+1] of a refined run at the coarse levels 0..N."""
    return np.ascontiguousarray(np.asarray(traces)[..., ::factor])


def crop_for_parity(w: Workload, shape, nt: int, max_rec: int = 64, seed: int = 0) -> Workload:
    """A small workload with the same physics/order/BC and the same kind of
    geometry, sized for the oracle: used by the parity tests."""
    rng = np.random.default_rng(seed)
    nd = len(shape)
    sl = tuple(slice(0, s) for s in shape)
    init = np.ascontiguousarray(np.asarray(w.init_param)[sl])
    true = None if w.true_param is None else np.ascontiguousarray(np.asarray(w.true_param)[sl])
    size = int(np.prod(shape))
    mid = [s // 2 for s in shape]
    mid[0] = min(2, shape[0] - 1)
    src = flat_index(shape, *mid)
    rec = np.sort(rng.choice(size, size=min(max_rec, size), replace=False)).astype(np.int64)
    return Workload(
        name=w.name + "_crop", shape=tuple(shape), h=w.h, order=w.order, bc=w.bc,
        physics=w.physics, true_param=true, init_param=init, vmax=w.vmax,
        cfl_fraction=w.cfl_fraction, sources=[src], receivers=[rec], nt=[nt], wavelet=w.wavelet,
        objective=w.objective, patch_sign=w.patch_sign)
