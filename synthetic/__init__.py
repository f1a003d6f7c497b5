"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds only input generation: cell sizes, ion lattices, plane-wave
orbital recipes, their periodic B-spline coefficient tables, Jastrow control
points, three-body Jastrow coefficients and initial electron positions. It performs none of the Monte Carlo
method's arithmetic (no orbital evaluation, no determinant, no Jastrow value,
no move), so both implementations can consume it without sharing method code.
"""
from .systems import (PRESETS, SystemSpec, build_inputs, spec_for, small_spec,
                      spline_coefficients, n_c_for, jastrow3_coefficients)

__all__ = ["PRESETS", "SystemSpec", "build_inputs", "spec_for", "small_spec",
           "spline_coefficients", "n_c_for", "jastrow3_coefficients"]
