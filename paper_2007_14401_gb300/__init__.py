"""GB300-native coupled guiding-center / Boris particle pusher (Bacchini et al. 2020).

Submodules:
  inputs  -- seeded synthetic workloads (fields on a periodic grid, particles)
  gcb     -- ctypes binding of the CUDA C-ABI library ``libgcb.so``
  build   -- compiles ``libgcb.so`` for sm_103a with nvcc

Importing the package does not load the CUDA library; ``gcb`` does, and it
raises if the library has not been built.
"""
__all__ = ["inputs", "gcb", "build"]
