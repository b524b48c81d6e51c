"""FP64 CPU oracle of the superposition adjoint method.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py, never by the product package.
"""
from .wave_oracle import *  # noqa: F401,F403
from .wave_oracle import (  # noqa: F401
    Medium, Shot, forward, adjoint, exact_gradient, superposition_gradient,
    misfit, adjoint_source, kernel_from_histories, auto_k, ricker, sine_burst,
    cfl_dt, stencil_weights, stencil_symbol_max, laplacian, divergence_operator,
    density_materials, patch_weight, SECOND_DERIVATIVE_WEIGHTS,
)
