"""libafminv: GB300-native (sm_103a) tip-sample force inversion for dynamic
AFM (after Busch, Zou & Ganapathysubramanian, arXiv 1109.0334).

Submodules:
  build      compile the CUDA library in-tree with nvcc
  afminv     ctypes binding of the C ABI (include/afminv.h)
  workloads  seeded synthetic workloads (inputs only)
"""
__all__ = ["build", "afminv", "workloads"]
