"""GB300-native particle-in-cell step for quantum plasmas (arXiv 2501.07465).

The compute path is libpic.so (CUDA kernels for sm_103a behind the C ABI of
include/pic.h); ``pic`` is its Python binding and ``inputs`` the seeded
workload generators.
"""
