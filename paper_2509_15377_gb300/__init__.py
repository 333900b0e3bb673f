"""GB300-native microscopic electron avalanche transport (arXiv:2509.15377).

csrc/        CUDA kernels for sm_103a and the C-ABI runtime (libgt_avalanche.so)
avalanche.py ctypes binding of include/gt_avalanche.h (no fallback path)
workloads.py seeded synthetic inputs (gases, fields, primaries)
build.py     in-tree nvcc build
"""
__all__ = ["avalanche", "workloads", "build"]
