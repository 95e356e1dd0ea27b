"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package only draws random numbers and lays out problem data (face
coefficients, sparsity patterns, right-hand sides).  It holds none of the
solver's arithmetic: no Krylov basis, Gram matrix, coordinate recurrence or
Ritz estimate is computed here.
"""
from .generators import (  # noqa: F401
    Stencil, CsrProblem, poisson2d_csr, varcoef_stencil, unit_stencil, rgg_laplacian_csr,
    random_rhs, uniform_vector, batched_stencils, config_problem, CONFIG_SEEDS,
)
