"""Seeded synthetic inputs for the MRHS Wilson-clover multigrid solver.

This package is the only code that both the FP64 oracle side (tests) and the
GPU side (tests, bench, smoke) use.  It holds no arithmetic of the solver:
it draws random gauge fields, random sources and random start vectors, and
nothing else.
"""
from .fields import (  # noqa: F401
    lattice_volume,
    site_index,
    site_coords,
    make_rng,
    gauge_unit,
    gauge_haar,
    gauge_exp,
    gaussian_field,
    gauge_transform_haar,
)
