"""GB300-native hot path of the Galilean electromagnetic PIC method (arXiv 2509.16793).

Submodules:
  workloads  seeded synthetic workloads (inputs only)
  gempic     ctypes binding of libgempic.so (the CUDA path behind the C-ABI)
  build      in-tree nvcc build of libgempic.so for sm_103a
"""
