"""Autotuner for the step kernel's tiling, with a JSON cache.

The tiling (`wave_model_set_tiling`: z-block depth, rows per CTA, ring
depth, pipeline) and the CTA launch order (`wave_model_set_schedule`) change
speed only, never results.  `tune()` times a short gradient call of the given
shots with each tiling candidate in the default (plane-major) order (CUDA
events inside libwave, `wave_timing_*`), keeps the fastest, times that tiling
once more in the other order, applies the faster and caches the choice under
a key of (dims, shape, order, physics, storage, Kahan, shots per launch).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

import torch

from . import wave as W

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json")


def candidates(ndim: int, nz: int, batched: bool = False):
    """Tilings worth timing: in 2D the rows per warp; in 3D the register-queue
    kernel (pipeline 3) for one field per launch, and for batched launches also
    the two-shots-per-pass kernel (4: cp.async staging; z-blocks of at most 32
    planes, 16 with Kahan compensation, keep the accumulator in tensor memory
    between the pairs) and the one-shot-at-a-time TMA kernel (5, z-block fixed
    at 8)."""
    if ndim == 2:
        return [(zb, 8, 3, 0) for zb in (8, 16, 32, 64, 128) if zb <= max(8, nz)]
    out = []
    for rows in (8, 16):
        for depth in (2, 3):
            for zb in (32, 64, 128):
                if zb <= max(32, nz):
                    out.append((zb, rows, depth, 3))
    if batched:
        out += [(zb, 16, 2, 4) for zb in (16, 32, 64, 128) if zb <= max(32, nz)]
        out += [(8, 16, 2, 5), (8, 16, 3, 5)]
    return out


def _key(model: W.Model, batch: int) -> str:
    return json.dumps([len(model.shape), list(model.shape), model.order, model.physics, model.storage,
                       bool(model.kahan), batch])


def _load() -> Dict[str, list]:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(cache: Dict[str, list]):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, CACHE)


def tune(model: W.Model, shots: Sequence[W.Shot], steps: int = 12, batched: bool = False,
         use_cache: bool = True, verbose: bool = False) -> tuple:
    """Pick and apply the fastest tiling for this model and shot set."""
    batch = len(shots) if batched else 1
    key = _key(model, batch)
    cache = _load() if use_cache else {}
    if key in cache:
        entry = list(cache[key])
        best = tuple(entry[:4])
        model.set_tiling(*best)
        model.set_schedule(entry[4] if len(entry) > 4 else 1)
        return best
    dev = model.param.device
    probe = []
    for s in (shots if batched else shots[:1]):
        n = min(steps, s.nt)
        probe.append(W.Shot(s.src, s.wavelet[:n + 1].contiguous(), s.rec,
                            None if s.observed is None else s.observed[:, :n + 1].contiguous()))
    nz = model.shape[0]

    def time_one(cand, order):
        model.set_tiling(*cand)
        model.set_schedule(order)
        model.gradient(probe, batched=batched, k=1.0)          # warm-up (and attribute setup)
        torch.cuda.synchronize(dev)
        W.timing_enable(True)
        model.gradient(probe, batched=batched, k=1.0)
        ms, n, _ = W.timing_read()
        W.timing_enable(False)
        if verbose:
            print(f"tiling {cand} order {order}: {ms / max(n, 1):.4f} ms per step launch")
        return ms / max(n, 1)

    results = [(time_one(cand, 1), cand) for cand in candidates(len(model.shape), nz, batched and batch > 1)]
    t_best, best = min(results)
    order = 1
    if len(model.shape) == 3 and best[3] in (3, 4) and time_one(best, 0) < t_best:
        order = 0
    model.set_tiling(*best)
    model.set_schedule(order)
    if use_cache:
        cache[key] = list(best) + [order]
        _save(cache)
    return best
