"""GB300-native particle-by-particle VMC/DMC hot path (tricubic B-spline orbitals,
Slater determinant ratios with Sherman-Morrison / delayed rank-k inverse updates,
B-spline Jastrow factors) behind the C ABI of ``include/qmcgb.h``.

The Python layer is a thin ctypes binding (``qmcgb``); the work runs in the CUDA
kernels of ``libqmcgb.so`` built from ``csrc/`` for sm_103a.
"""
from .qmcgb import (QMCError, System, Walkers, load, system_from_inputs)  # noqa: F401

__all__ = ["QMCError", "System", "Walkers", "load", "system_from_inputs"]
