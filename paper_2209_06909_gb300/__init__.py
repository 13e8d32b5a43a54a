"""GB300-native Multiway Powersort (arXiv 2209.06909).

The sort runs entirely in hand-written CUDA kernels for sm_103a behind the C
ABI declared in ``include/mps.h`` (``libmps.so``).  ``paper_2209_06909_gb300.mps``
is the thin ctypes binding; ``inputs`` holds the seeded synthetic workloads.
"""
