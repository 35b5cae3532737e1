"""Uniform sampling without replacement (Sec. 3.2 "Sampling and interpolation", Eq. 4).

Test infrastructure only.  The paper draws n indices Omega uniformly at
random from {1..N} without replacement and defines M_ij = 1 iff j = omega_i.
Reading (integer only, so both sides agree bit for bit): node i gets the key
k_i = output i of SplitMix64 seeded with ``seed``; Omega is the n nodes with
the smallest (k_i, i) in lexicographic order, returned sorted by node id.
Since the keys are i.i.d. uniform 64-bit words, every n-subset is equally
likely (ties between keys are broken by index and have probability ~2^-64).

Pins (tests/test_oracle_sampling.py): exactly n distinct sorted indices;
inclusion frequency n/N per node over many seeds (chi-square); n = N returns
every node; the sampling matrix of Eq. 4 has one 1 per row.
"""
from __future__ import annotations

import numpy as np

from .rng import splitmix64_at


def sample_keys(n_nodes: int, seed: int) -> np.ndarray:
    return splitmix64_at(seed, np.arange(n_nodes, dtype=np.uint64))


def sample(n_nodes: int, n: int, seed: int) -> np.ndarray:
    """Omega as int64[n], sorted ascending."""
    if n < 0 or n > n_nodes:
        raise ValueError("need 0 <= n <= N")
    keys = sample_keys(n_nodes, seed)
    order = np.lexsort((np.arange(n_nodes), keys))  # primary key, then index
    return np.sort(order[:n]).astype(np.int64)


def sampling_matrix(n_nodes: int, omega: np.ndarray) -> np.ndarray:
    """Dense M of Eq. 4 (small cases only)."""
    m = np.zeros((len(omega), n_nodes))
    m[np.arange(len(omega)), omega] = 1.0
    return m
