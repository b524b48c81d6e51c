"""GB300-native memory-efficient adjoint (superposition) wave-equation gradients.

The compute path is the C-ABI library ``libwave.so`` (hand-written sm_103a CUDA
kernels, declared in ``include/wave.h``); ``paper_2509_15744_gb300.wave`` is
the thin ctypes binding over it and ``paper_2509_15744_gb300.autograd`` the
torch.autograd.Function wrapper.  Importing the binding fails loudly when the
library has not been built.
"""
__version__ = "0.1.0"
