"""GB300-native generalized-harmonic (GH) shell evolution (arXiv:1804.09101 hot path).

Submodules:
  gh         ctypes binding of the C-ABI library libgh.so (include/gh.h)
  workloads  synthetic workload shapes and seeded input generators
  build      in-tree nvcc build of libgh.so for sm_103a
  costmodel  the paper's operation-count models (Secs. 3.3 and 3.4)
"""
