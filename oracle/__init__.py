"""FP64 CPU oracle for similarity-based fuzzy clustering (test infrastructure).

This package is test infrastructure only.  It is a plain, slow, obviously
correct restatement of what the paper computes, in float64 with numpy and
scipy.sparse, written step by step in the paper's order and notation.  Only
the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it; the CUDA library never calls it and shares no code with it.

Notation: the paper's membership matrix X (C x N, columns on the simplex) is
handled here as U = X^T (N x C, rows on the simplex), so n = N and k = C.

Parity status: every function is pinned by the non-GPU tests (closed forms,
brute force, the paper's 7-node example, invariants of Theorem 2.1); none is
"parity unpinned".
"""
from .fista import (
    frob2,
    objective_dense,
    objective_trace,
    loss_terms,
    gradient_matrix,
    gradient_columns,
    hessian_apply,
    hessian_apply_sparse,
    curvature,
    slope,
    duchi,
    project_omega,
    lipschitz,
    gpa,
    fista,
    OracleResult,
    csr_from_edges,
    spectral_norm,
    momentum_factors,
    fista_step_rows,
    gram_blocks,
)

__all__ = [
    "frob2", "objective_dense", "objective_trace", "loss_terms", "gradient_matrix", "gradient_columns",
    "hessian_apply", "hessian_apply_sparse", "curvature", "slope", "duchi", "project_omega", "lipschitz", "gpa", "fista",
    "OracleResult", "csr_from_edges", "spectral_norm", "momentum_factors", "fista_step_rows",
    "gram_blocks",
]
