"""Seeded synthetic workloads for C = A·B (CSR operands).

This package only draws inputs: matrices, value arrays and seeds.  It holds
none of the SpGEMM arithmetic, so both the CPU oracle and the GPU path take
their inputs from here without sharing any of the method's code.

The shapes and value distributions stand in for the paper's test problems
(Section 4: A×A products of UF-collection matrices and multigrid R×A×P
triple products), which are not available here.
"""

from .csr import Csr, csr_from_coo, shuffle_rows, identity, permutation_matrix, lower_triangle
from .gen import (
    laplace2d_5pt,
    stencil3d_27pt,
    laplace3d_7pt,
    aggregation,
    rmat_symmetric,
    batched_pairs,
    batched_fresh_values,
    random_csr,
    values_on_pattern,
    config_workload,
)

__all__ = [
    "Csr", "csr_from_coo", "shuffle_rows", "identity", "permutation_matrix", "lower_triangle",
    "laplace2d_5pt", "stencil3d_27pt", "laplace3d_7pt", "aggregation",
    "rmat_symmetric", "batched_pairs", "batched_fresh_values", "random_csr",
    "values_on_pattern", "config_workload",
]
