"""Observed data from a refined grid (the paper's guard against the inverse
crime: data on a 2x grid with 2x steps).  The refinement map of
`workloads.refined` (node positions, Kronecker source scaling factor^d,
wavelet sampled at the fine step, coarse levels every factor-th fine level) is
checked with the oracle: traces converge at second order under refinement, so
a wrong scaling, position or time sampling shows up as a broken rate."""
import numpy as np
import pytest

import oracle as O
from paper_2509_15744_gb300 import workloads as WL


def base_workload():
    n = 48
    shape = (n, n)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v = (2000.0 + 300.0 * np.exp(-((yy - 30.0) ** 2 + (xx - 26.0) ** 2) / 60.0)).astype(np.float32)
    src = WL.flat_index(shape, 24, 20)
    rec = np.array([WL.flat_index(shape, 24, 24), WL.flat_index(shape, 20, 22), WL.flat_index(shape, 28, 18)])
    return WL.Workload(name="smooth48", shape=shape, h=20.0, order=2, bc="dirichlet", physics="velocity",
                       true_param=v, init_param=v, vmax=2300.0, cfl_fraction=0.5, sources=[src],
                       receivers=[rec], nt=[70], wavelet=WL.WaveletSpec("ricker", 8.0))


def traces(w):
    dt = O.cfl_dt(w.h, w.vmax, w.ndim, w.order, w.cfl_fraction)
    med = O.Medium(w.physics, w.true_param.astype(np.float64), w.h, dt, w.order, w.bc)
    t = np.arange(w.nt[0] + 1) * dt
    wav = w.wavelet.psi0 * O.ricker(t, w.wavelet.freq)
    shot = O.Shot(w.sources[0], wav, w.receivers[0], None, 1.0)
    return O.forward(med, shot, w.nt[0])["traces"], dt


def test_refinement_map():
    w = base_workload()
    r = WL.refined(w, 2)
    assert r.shape == (96, 96) and r.h == 10.0 and r.nt == [140]
    assert r.wavelet.psi0 == 4.0 and r.wavelet.freq == w.wavelet.freq
    assert r.sources == [WL.flat_index(r.shape, 48, 40)]
    assert list(r.receivers[0]) == [WL.flat_index(r.shape, 48, 48), WL.flat_index(r.shape, 40, 44),
                                    WL.flat_index(r.shape, 56, 36)]
    # the model keeps its value at every coarse node
    assert (r.true_param[::2, ::2] == w.true_param).all()
    # the time step halves with the grid spacing (same fraction of the limit)
    dt = O.cfl_dt(w.h, w.vmax, 2, 2, 0.5)
    assert O.cfl_dt(r.h, r.vmax, 2, 2, 0.5) == pytest.approx(dt / 2)


def test_refined_traces_converge_at_second_order():
    w = base_workload()
    t1, _ = traces(w)
    t2f, _ = traces(WL.refined(w, 2))
    t4f, _ = traces(WL.refined(w, 4))
    t2 = WL.coarse_samples(t2f, 2)
    t4 = WL.coarse_samples(t4f, 4)
    assert t2.shape == t1.shape == t4.shape
    e1 = np.linalg.norm(t1 - t4)
    e2 = np.linalg.norm(t2 - t4)
    # T_h - T_ref ~ C h^2: (1 - 1/16) / (1/4 - 1/16) = 5
    assert 3.5 < e1 / e2 < 7.0, e1 / e2
    assert e2 < 0.1 * np.linalg.norm(t4)


def test_unscaled_fine_source_is_caught():
    # planted mistake: a fine-grid Kronecker source without the factor^d scaling
    w = base_workload()
    r = WL.refined(w, 2)
    r.wavelet = WL.WaveletSpec(r.wavelet.kind, r.wavelet.freq, r.wavelet.nc, 1.0)
    t1, _ = traces(w)
    t2 = WL.coarse_samples(traces(r)[0], 2)
    assert np.linalg.norm(t2 - t1) > 0.5 * np.linalg.norm(t1)
