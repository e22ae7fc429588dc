"""Seeded synthetic linear systems shaped like the paper's workloads.

This package only builds inputs (CSR matrices, right-hand sides, targets).
It holds none of the solver's arithmetic and is shared by the CPU oracle,
the tests and the benchmark.
"""
from .generators import (  # noqa: F401
    CSR, stencil2d, stencil3d_convdiff, vardiff3d, aniso2d, random_band,
    diagonal, jacobi_chain, rhs_from_solution, uniform_vector, config_c1, config_c2,
    config_c3, config_c4, config_c5, CONFIGS,
)
