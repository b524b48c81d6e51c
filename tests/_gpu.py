"""GPU-side construction of the shared test problems (tests/_problems.py):
the model and shots in libwave's binding.  Inputs only; no arithmetic."""
from __future__ import annotations

import numpy as np
import torch

DEV = "cuda"


def gpu_model(W, prob, param=None, **kw):
    p = prob.param0 if param is None else param
    return W.Model(torch.from_numpy(np.ascontiguousarray(p)).to(DEV), prob.h, prob.dt, prob.order, prob.physics,
                   prob.bc, **kw)


def gpu_shots(W, prob, with_observed=True):
    shots = []
    for i in range(len(prob.src)):
        if prob.wavelets is not None:
            wav = torch.from_numpy(prob.wavelets[i]).to(DEV)
        else:
            wav = W.wavelet(prob.wav_kind, prob.wav_freq, prob.dt, prob.nt[i], device=DEV)
        obs = None
        if with_observed and prob.observed is not None and prob.observed[i] is not None:
            obs = torch.from_numpy(prob.observed[i]).to(DEV)
        shots.append(W.Shot(prob.src[i], wav, torch.from_numpy(prob.rec[i]).to(DEV), obs))
    return shots
