"""GB300-native (sm_103a) hot path of MPI-AMRVAC (arXiv:2004.03275).

Modules:
  amrvac  -- Python binding of the C ABI in include/amrvac_gb300.h (CUDA only)
  inputs  -- seeded synthetic initial conditions
  build   -- in-tree nvcc build of libamrvac_gb300.so
Nothing is loaded at import time.
"""
__all__ = ["amrvac", "inputs", "build"]
