"""GB300-native Galilean-PSATD particle-in-cell step (Kirchen et al., arXiv:1608.00215).

The compute path is the CUDA library ``libgalpic.so`` (C ABI in
``include/galpic.h``); ``paper_1608_00215_gb300.galpic`` is its ctypes
binding, with the same function names, and ``Sim`` a thin owner of one run's
device workspace. Importing the binding raises if the library is missing:
there is no CPU fallback.
"""
__all__ = ["galpic"]
