"""GB300 (sm_103a) KADABRA sampling: the hot path of arXiv 1903.09422's case study.

Modules:
  kad    -- Python binding of the C ABI in include/kad.h (libkad.so, CUDA kernels)
  gen    -- seeded synthetic graph inputs (R-MAT, grid + shortcuts, hyperbolic, ER)
  build  -- in-tree nvcc build of libkad.so
"""
__all__ = ["kad", "gen", "build"]
