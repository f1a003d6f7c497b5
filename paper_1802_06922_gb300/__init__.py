"""GB300-native particle-by-particle VMC/DMC hot path (tricubic B-spline orbitals,
Slater determinant ratios with Sherman-Morrison / delayed rank-k inverse updates,
B-spline Jastrow factors) behind the C ABI of ``include/qmcgb.h``.

The Python layer is a thin ctypes binding (``qmcgb``); the work runs in the CUDA
kernels of ``libqmcgb.so`` built from ``csrc/`` for sm_103a.
"""
from .qmcgb import (DMC, QMCError, System, Walkers, load, measure_rates,  # noqa: F401
                    slater_invert, slater_invert_noalloc, system_from_inputs)
from .autotune import tune_delay, tune_launch  # noqa: F401

__all__ = ["DMC", "QMCError", "System", "Walkers", "load", "measure_rates", "slater_invert",
           "slater_invert_noalloc", "system_from_inputs", "tune_delay", "tune_launch"]
