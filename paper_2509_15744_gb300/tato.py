"""Design chain of the transient acoustic topology optimisation (Sec. 5.2,
'Constraints'; Sec. 6.2): the indicator gamma is filtered (density filter
with linear decay), projected (smooth Heaviside with beta-continuation) and
clipped to [0, 1] before it enters the wave model, and Adam updates gamma
with the chain rule of that map.

These are torch operations on the device around the autograd Function
`wave_misfit`, whose gradient is the memory-efficient adjoint sensitivity of
libwave; torch's autograd supplies the transposed filter and the projection
derivative of the chain rule.

    problem = WaveProblem(h, dt, shots, physics="density", bc="neumann",
                          objective="patch", patch_sign=+1)
    gamma, history = optimise(gamma0, problem, iterations=50)
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Tuple

import torch
import torch.nn.functional as F

from .autograd import WaveProblem, wave_misfit


def filter_kernel(rf: float, ndim: int, dtype=torch.float32, device=None) -> torch.Tensor:
    """Weights w(x) = rf - |x| of the grid offsets with |x| < rf (linear decay),
    as a (2r+1)^ndim tensor, r = ceil(rf) - 1."""
    if rf <= 0.0:
        raise ValueError("filter radius must be positive")
    r = int(math.ceil(rf)) - 1
    ax = torch.arange(-r, r + 1, dtype=torch.float64)
    grids = torch.meshgrid(*([ax] * ndim), indexing="ij")
    dist = torch.sqrt(sum(g * g for g in grids))
    w = torch.where(dist < rf, rf - dist, torch.zeros_like(dist))
    return w.to(dtype=dtype, device=device)


def density_filter(gamma: torch.Tensor, rf: float) -> torch.Tensor:
    """gamma~_i = sum_k w(x_i - x_k) gamma_k / sum_k w(x_i - x_k) over the
    neighbours k of i inside the grid (|x_i - x_k| < rf)."""
    nd = gamma.dim()
    if nd not in (2, 3):
        raise ValueError("gamma must be a 2D or 3D grid")
    k = filter_kernel(rf, nd, gamma.dtype, gamma.device)
    r = (k.shape[0] - 1) // 2
    conv = F.conv2d if nd == 2 else F.conv3d
    x = gamma[None, None]
    num = conv(x, k[None, None], padding=r)
    den = conv(torch.ones_like(x), k[None, None], padding=r)
    return (num / den)[0, 0]


def heaviside_projection(x: torch.Tensor, beta: float, eta: float = 0.5) -> torch.Tensor:
    """Smooth Heaviside H(x) = (tanh(beta eta) + tanh(beta (x - eta))) /
    (tanh(beta eta) + tanh(beta (1 - eta)))."""
    te = math.tanh(beta * eta)
    return (te + torch.tanh(beta * (x - eta))) / (te + math.tanh(beta * (1.0 - eta)))


def beta_schedule(iteration: int, beta0: float = 1.0, factor: float = 1.1, every: int = 5) -> float:
    """beta-continuation: beta0, raised by `factor` every `every` iterations."""
    return beta0 * factor ** (iteration // every)


def design(gamma: torch.Tensor, rf: float, beta: float, eta: float = 0.5) -> torch.Tensor:
    """Filtered, projected and clipped indicator that enters the wave model."""
    return heaviside_projection(density_filter(gamma, rf), beta, eta).clamp(0.0, 1.0)


def optimise(gamma0: torch.Tensor, problem: WaveProblem, iterations: int, lr: float = 0.1, rf: float = 1.5,
             eta: float = 0.5, eps: float = 1e-5, normalise: bool = True,
             callback: Optional[Callable[[int, float, torch.Tensor], None]] = None
             ) -> Tuple[torch.Tensor, List[float]]:
    """Adam on gamma (learning rate lr), gamma clipped to [eps, 1] after each
    update; returns the final gamma and the objective of each iteration.

    normalise: Adam descends C / |C_0| (C_0 the first objective), which has the
    same minimiser; without it a patch energy of order 1e-20 gives gradients
    far below Adam's epsilon and the steps vanish."""
    if problem.physics != "density":
        raise ValueError("the design chain acts on the density form (gamma)")
    gamma = torch.nn.Parameter(gamma0.detach().clone().to(torch.float32))
    opt = torch.optim.Adam([gamma], lr=lr)
    history: List[float] = []
    scale = None
    for it in range(iterations):
        beta = beta_schedule(it)
        opt.zero_grad(set_to_none=True)
        c = wave_misfit(design(gamma, rf, beta, eta).contiguous(), problem)
        if scale is None:
            c0 = abs(float(c.item()))
            scale = 1.0 / c0 if (normalise and c0 > 0.0) else 1.0
        (c * scale).backward()
        opt.step()
        with torch.no_grad():
            gamma.clamp_(eps, 1.0)
        history.append(float(c.item()))
        if callback is not None:
            callback(it, history[-1], gamma)
    return gamma.detach(), history
