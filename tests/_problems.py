"""Shared construction of matching oracle / GPU problems for the tests.

Inputs come from seeded generators (numpy) and the oracle; nothing here takes
a value from the CUDA path.  Each side builds its own wavelet samples from the
same parameters (the GPU with wave_wavelet, the oracle with its own formula)
unless a test passes explicit samples.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

import oracle as O


@dataclass
class Problem:
    physics: str
    order: int
    bc: str
    shape: tuple
    h: float
    dt: float
    nt: List[int]
    param0: np.ndarray                  # float32 model at which things are evaluated
    param_true: Optional[np.ndarray]    # float32 model of the observed data
    src: List[int]
    rec: List[np.ndarray]
    wav_kind: str
    wav_freq: float
    objective: str = "l2"
    patch_sign: float = 1.0
    wavelets: Optional[List[np.ndarray]] = None   # explicit samples (float32) if given
    observed: Optional[List[Optional[np.ndarray]]] = None

    def medium(self, param=None):
        p = self.param0 if param is None else param
        return O.Medium(self.physics, p.astype(np.float64), self.h, self.dt, self.order, self.bc)

    def oracle_wavelet(self, i):
        if self.wavelets is not None:
            return self.wavelets[i].astype(np.float64)
        t = np.arange(self.nt[i] + 1) * self.dt
        if self.wav_kind == "ricker":
            return O.ricker(t, self.wav_freq)
        return O.sine_burst(t, self.wav_freq, 2, 1.0)

    def weight(self, i):
        if self.objective == "l2":
            return 1.0
        return O.patch_weight(len(self.rec[i]), self.patch_sign)

    def oracle_shots(self):
        out = []
        for i in range(len(self.src)):
            obs = None if self.observed is None or self.observed[i] is None else self.observed[i].astype(np.float64)
            out.append(O.Shot(self.src[i], self.oracle_wavelet(i), self.rec[i], obs, self.weight(i)))
        return out


def make_problem(shape, order=2, bc="dirichlet", physics="velocity", nt=100, nrec=24, seed=0,
                 objective="l2", nshots=1, random_wavelet=False, patch=None, src=None, rec=None,
                 nt_list=None, patch_sign=1.0):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    size = int(np.prod(shape))
    if physics == "velocity":
        h = 10.0
        true = rng.uniform(1800.0, 3200.0, shape).astype(np.float32)
        p0 = np.full(shape, 2500.0, np.float32)
        p0 += rng.uniform(-200, 200, shape).astype(np.float32)
        vmax = max(float(true.max()), float(p0.max()))
        dt = O.cfl_dt(h, vmax, nd, order, 0.5)
        kind, freq = "ricker", 1.0 / (25 * dt)
    else:
        h = 2e-3
        true = rng.uniform(0.1, 1.0, shape).astype(np.float32)
        p0 = rng.uniform(0.1, 1.0, shape).astype(np.float32)
        dt = O.cfl_dt(h, 509.8366, nd, 2, 0.5)
        kind, freq = "sine_burst", 1.0 / (30 * dt)
    nts = list(nt_list) if nt_list is not None else [nt] * nshots
    srcs, recs = [], []
    for s in range(nshots):
        if src is not None:
            srcs.append(int(src[s] if isinstance(src, (list, tuple)) else src))
        else:
            c = [int(rng.integers(0, n)) for n in shape]
            c[0] = min(2, shape[0] - 1)
            srcs.append(int(np.ravel_multi_index(tuple(c), shape)))
        if rec is not None:
            recs.append(np.asarray(rec, np.int64))
        elif patch is not None:
            recs.append(np.asarray(patch, np.int64))
        else:
            recs.append(np.sort(rng.choice(size, size=min(nrec, size), replace=False)).astype(np.int64))
    wavs = None
    if random_wavelet:
        wavs = [rng.standard_normal(n + 1).astype(np.float32) for n in nts]
    prob = Problem(physics, order, bc, tuple(shape), h, dt, nts, p0, true, srcs, recs, kind, freq,
                   objective=objective, patch_sign=patch_sign, wavelets=wavs)
    if objective == "l2":
        med_true = prob.medium(true)
        obs = []
        for i in range(nshots):
            tr = O.forward(med_true, O.Shot(srcs[i], prob.oracle_wavelet(i), recs[i]), nts[i])["traces"]
            obs.append(tr.astype(np.float32))
        prob.observed = obs
    return prob


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
