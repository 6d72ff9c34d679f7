"""GB300 (sm_103a) staggered-fermion RHMC hot path: the C-ABI library libstag
(CUDA kernels in csrc/, header in include/stag.h) and its thin ctypes
binding (stag.py).  Importing the package does not load the library; the
first call into `stag` does, and fails loudly if it has not been built."""
__all__ = ["stag", "build"]
