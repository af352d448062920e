"""GB300-native batched Kerr geodesic integration (arXiv:1706.07062 hot path).

The compute lives in libkerr.so (CUDA, sm_103a) behind the C ABI of
include/kerr.h; ``kerr`` is its thin ctypes binding and ``workloads`` holds
the seeded synthetic input generators.
"""
from . import kerr  # noqa: F401
