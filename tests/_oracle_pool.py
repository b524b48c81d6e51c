"""Oracle runs spread over host cores for the larger parity tests.

The workers import only numpy and the oracle.  The pool is created with the
'spawn' start method, which is safe after the parent process has initialised
CUDA (a forked child of such a process can hang).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

import oracle as O


def _medium(spec):
    physics, param, h, dt, order, bc = spec
    return O.Medium(physics, np.asarray(param, np.float64), h, dt, order, bc)


def forward_traces(job):
    """Traces [nrec, nt+1] of one shot (FP64)."""
    spec, src, wav, rec, nt = job
    return O.forward(_medium(spec), O.Shot(src, np.asarray(wav, np.float64), np.asarray(rec)), nt)["traces"]


def adjoint_source_of(job):
    """f_adj of one shot at the model of `spec` (Eq. adjointSource1)."""
    spec, src, wav, rec, nt, obs, weight = job
    shot = O.Shot(src, np.asarray(wav, np.float64), np.asarray(rec), obs, weight)
    tr = O.forward(_medium(spec), shot, nt)["traces"]
    return O.adjoint_source(tr, shot, nt)


def superposition(job):
    """(K_tilde, C) of Algorithm 1 for one shot at the given k."""
    spec, src, wav, rec, nt, obs, weight, k = job
    shot = O.Shot(src, np.asarray(wav, np.float64), np.asarray(rec), obs, weight)
    r = O.superposition_gradient(_medium(spec), [shot], nt, k)
    return r["K_tilde"], r["C"]


def exact_gradient_of(job):
    """(grad, C) of the stored-history adjoint for one shot (Sec. 2.2)."""
    spec, src, wav, rec, nt, obs, weight = job
    shot = O.Shot(src, np.asarray(wav, np.float64), np.asarray(rec), obs, weight)
    c, g, _ = O.exact_gradient(_medium(spec), [shot], nt)
    return g, c


def pool(nproc=None):
    n = nproc or min(16, os.cpu_count() or 1)
    return mp.get_context("spawn").Pool(n)


def superposition_many(job):
    """(K_tilde, C) of Algorithm 1 summed over several shots of one record
    length, at the given k: job = (spec, [(src, wav, rec, obs, weight)], nt, k)."""
    spec, shots, nt, k = job
    osh = [O.Shot(s, np.asarray(w, np.float64), np.asarray(r), o, wt) for s, w, r, o, wt in shots]
    res = O.superposition_gradient(_medium(spec), osh, nt, k)
    return res["K_tilde"], res["C"]


def k0_of(job):
    """k = ||psi|| / ||f_adj|| (the automatic rule at ratio 1) of one shot:
    job = (spec, (src, wav, rec, obs, weight), nt)."""
    spec, (s, w, r, o, wt), nt = job
    shot = O.Shot(s, np.asarray(w, np.float64), np.asarray(r), o, wt)
    tr = O.forward(_medium(spec), shot, nt)["traces"]
    return O.auto_k(shot, O.adjoint_source(tr, shot, nt), nt, 1.0)
