"""GB300-native BSPAI-GMRES-IR (Khan & Carson, arXiv 2307.03914).

Submodules:
  workloads  seeded synthetic inputs (no method arithmetic)
  bspai      ctypes binding of the CUDA library libbspai.so (C-ABI in include/bspai.h)
  build      nvcc build of the library for sm_103a
"""
__all__ = ["workloads", "bspai", "build"]
