"""Seeded synthetic inputs for the HLBM NACA 0012 cases.

This module builds geometry only: the analytic NACA 0012 surface, a body-fitted
O-type triangular mesh bounded by an ellipse, the nested Cartesian level boxes
and the inner interface (hole) ellipse.  It holds none of the method's
arithmetic (no equilibria, no finite-volume coefficients, no interpolation
weights); both the CUDA library and the CPU oracle receive the same arrays
from here and do their own set-up from them.
"""
from .naca import (  # noqa: F401
    CONFIGS,
    ENSEMBLE_SIZES,
    Case,
    ensemble,
    ensemble_case,
    make_case,
    naca0012_half_thickness,
    o_mesh,
    patch_case,
    square_patch,
    thickness_modes,
    uniform_equivalent,
)
