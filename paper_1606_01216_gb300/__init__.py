"""GB300-native (sm_103a) shifted-system solve path of arXiv 1606.01216.

Sequences of shifted sparse SPD systems (s^2 M + s D + K) X = F with
proportional damping D = alpha M + beta K, solved by SPAI-preconditioned CG,
with SPAI construction and the SPAI update from one shift to the next.

Submodules:
  workloads  seeded synthetic beam inputs (no method arithmetic)
  airga      ctypes binding of the C-ABI library libairga.so (CUDA kernels)
  build      nvcc build of libairga.so
"""
__all__ = ["workloads", "airga", "build"]
