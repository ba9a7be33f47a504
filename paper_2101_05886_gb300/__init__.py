"""GB300 implementation of the free-stream-preserving upwind finite-difference
residual (arXiv 2101.05886).

Submodules:
  inputs   seeded grids and initial states (numpy only)
  binding  ctypes binding of libfpgb300.so (the C ABI of include/fp.h)
  solver   Block / Batch wrappers over the binding for torch tensors
  build    nvcc build of libfpgb300.so (sm_103a)
"""
