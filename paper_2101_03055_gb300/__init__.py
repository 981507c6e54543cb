"""GB300 (sm_103a) lattice Boltzmann solver for the coupled cross-diffusion-fluid
system of Zhan, Chai & Shi (arXiv:2101.03055).

  build   -- compiles the CUDA library libcdflb.so in-tree with nvcc
  lib     -- ctypes binding of the C ABI (include/cdf_lb.h) and `Solver`
  inputs  -- seeded synthetic problems and initial fields

Importing the package loads nothing; `lib.load()` (called by every binding)
raises if the CUDA library is missing.
"""
__all__ = ["build", "lib", "inputs"]
