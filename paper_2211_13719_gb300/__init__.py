"""GB300-native MRHS multigrid solver for the Wilson-clover Dirac equation.

The hot path (fine hopping + clover stencil, coarse 9-point stencil,
restriction / prolongation, batched inner products, V-cycle, mixed-precision
FGMRES, continuous-batching server) lives in the CUDA library built from
``csrc/`` and is reached through the C ABI of ``include/mrhs.h``; ``mrhs``
is its ctypes binding.
"""
from . import mrhs  # noqa: F401
