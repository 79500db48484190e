"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds no arithmetic of the clustering method: it only draws
graphs (edge lists, CSR similarity matrices with a unit diagonal) and
Dirichlet(1) starting memberships from a counter-based generator, so that the
oracle and the GPU path can be fed identical inputs.
"""
from .rng import hash_u64, uniform01, stream_key
from .gen import (
    sbm_pairs,
    dcsbm_edges,
    two_cluster_er_edges,
    two_cluster_graph,
    second_row_start,
    assemble_csr,
    pair_weights,
    dirichlet_u0,
    GraphSpec,
    make_graph,
    batch_specs,
)

__all__ = [
    "hash_u64", "uniform01", "stream_key",
    "sbm_pairs", "dcsbm_edges", "two_cluster_er_edges", "two_cluster_graph", "second_row_start",
    "assemble_csr", "pair_weights", "dirichlet_u0", "GraphSpec", "make_graph", "batch_specs",
]
