"""B300-native explicit finite-volume shallow-water step (BASEMENT v3 hydrodynamics).

Submodules:
  bm         -- ctypes binding of the C ABI in include/bm.h (libbm.so, CUDA sm_103a)
  build      -- nvcc build of libbm.so in-tree
  workloads  -- seeded synthetic meshes and states
"""
