"""GB300-native moving-boundary lattice electrokinetics (Kuron et al., arXiv 1607.04572).

The compute path is libek.so (hand-written CUDA for sm_103a behind the C ABI
of include/ek.h); ``paper_1607_04572_gb300.ek`` is its ctypes binding.
"""
from . import ek  # noqa: F401
from .ek import EKSystem, EKError, load_library  # noqa: F401
