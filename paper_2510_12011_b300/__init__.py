"""B300-native monodomain hot path (TorchCor, arXiv 2510.12011).

  paper_2510_12011_b300.tc       ctypes binding of the C ABI (include/tc.h)
  paper_2510_12011_b300.inputs   seeded synthetic meshes and workloads
  paper_2510_12011_b300.build    nvcc build of csrc/ into lib/libtc_b300.so
"""
__all__ = ["tc", "inputs", "build"]
