"""GB300 (sm_103a) domain-decomposition solver for the Wilson-clover Dirac equation.

The compute path is the C-ABI library libdd.so (CUDA kernels); `dd` is a thin ctypes
binding with the same function names as include/dd.h.
"""
from .dd import *  # noqa: F401,F403
