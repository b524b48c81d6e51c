"""torch.autograd wrapper: model grid in, misfit out, gradient from libwave.

Algorithm 1 produces the cost C and the sensitivity K~ in the same pass
(Sec. 4), so the forward of the Function runs the whole superposition
gradient and keeps K~; backward only scales it by the incoming gradient.
All arithmetic of the path runs in libwave's kernels.

    problem = WaveProblem(h=10.0, dt=dt, order=8, shots=[...])
    v = torch.nn.Parameter(v0)              # velocity grid [m/s] on cuda
    C = wave_misfit(v, problem)             # FP64 scalar
    C.backward()                            # v.grad = dC/dv (superposition)
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import torch

from . import wave as W


@dataclass
class WaveProblem:
    h: float
    dt: float
    shots: List[W.Shot]
    order: int = 2
    physics: str = "velocity"
    bc: str = "dirichlet"
    storage: str = "f32"
    kahan: bool = False
    objective: str = "l2"
    patch_sign: float = 1.0
    k: Optional[float] = None
    k_ratio: Optional[float] = None
    batched: bool = False
    mode: str = "superposition"
    last_k: Optional[float] = field(default=None, init=False)
    # the model is built (with its one host wait, the stability check) on the
    # first call and receives later parameters without a wait; model.check()
    # reports an unstable or non-finite parameter
    model: Optional[W.Model] = field(default=None, init=False, repr=False)


class WaveGradient(torch.autograd.Function):
    """C(param) with dC/dparam from the memory-efficient adjoint (Algorithm 1).

    param: velocity [m/s] (velocity form) or gamma (density form), float32
    CUDA tensor.  The gradient is with respect to param itself (the dC/dv
    chain rule m = 1/v^2 runs in the finish kernel)."""

    @staticmethod
    def forward(ctx, param: torch.Tensor, problem: WaveProblem):
        p = param.detach().contiguous()
        model = problem.model
        key = (tuple(p.shape), p.device, problem.h, problem.dt, problem.order, problem.physics, problem.bc,
               problem.storage, problem.kahan)
        if model is None or getattr(model, "_problem_key", None) != key:
            model = W.Model(p, problem.h, problem.dt, problem.order, problem.physics, problem.bc,
                            storage=problem.storage, kahan=problem.kahan)
            model._problem_key = key
            problem.model = model
        else:
            model.set_param(p)
        grad, mis, kd = model.gradient(problem.shots, objective=problem.objective, k=problem.k,
                                       k_ratio=problem.k_ratio, mode=problem.mode, batched=problem.batched,
                                       grad_wrt="param", patch_sign=problem.patch_sign)
        problem.last_k = kd
        ctx.save_for_backward(grad)
        return mis.reshape(())

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad * grad_out.to(grad.dtype), None


def wave_misfit(param: torch.Tensor, problem: WaveProblem) -> torch.Tensor:
    """Misfit C (FP64 scalar tensor) differentiable with respect to param."""
    return WaveGradient.apply(param, problem)
