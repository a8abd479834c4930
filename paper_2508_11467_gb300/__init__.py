"""GB300-native bidiagonal divide-and-conquer SVD (sm_103a CUDA behind a C ABI).

The compute path lives in ``csrc/`` (CUDA kernels + the ``extern "C"`` entry
points declared in ``include/bdc.h``) and is reached through the thin ctypes
binding in :mod:`paper_2508_11467_gb300.bdc`.  Importing the package does not
load the library; the first call does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "bdc"]
