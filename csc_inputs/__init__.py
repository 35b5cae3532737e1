"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds input generation only: random graphs in CSR form (the
stochastic block model and Chung-Lu power-law graphs of the paper's
experiments, Sec. 5.1 and the supplementary heterogeneous SBM) and seeded
Gaussian signal blocks.  It contains none of the clustering method's
arithmetic, so both the CUDA path and the CPU oracle can consume it without
sharing any computation.
"""
from .graphs import (  # noqa: F401
    CSRGraph,
    sbm,
    sbm_probabilities,
    epsilon_c,
    chung_lu,
    chung_lu_weights,
    from_edges,
    ring,
    complete,
    disjoint_cliques,
    complete_bipartite,
    path,
    erdos_renyi,
    block_diagonal,
)
from .signals import gaussian_block, score_profile, workload_sizes  # noqa: F401
from .datasets import bracket_graph, batched_sbm_set  # noqa: F401
