"""Seeded synthetic workloads shaped like the paper's solids (2-atom fcc cells,
large uncontracted Gaussian bases, Gamma-centred k-meshes).

This package is shared by the CPU oracle and the GPU path. It holds only input
preparation -- geometry, basis definition, k-point lists and seeded orbital
coefficients -- and none of the exchange-build arithmetic (no AO-on-grid
evaluation, no FFT, no kernel, no contraction).
"""
from .synthetic import (  # noqa: F401
    BOHR_PER_ANGSTROM,
    Workload,
    fcc_cell,
    geometric_exponents,
    make_shells,
    gamma_mesh,
    random_coefficients,
    analytic_overlap,
    lowdin_orthonormalize,
    config,
    config_names,
    small_workload,
)
