"""Seeded graph collections: the learned lambda_k-bracket set and the batched set.

``bracket_graph(i)`` draws graph i of the bracket-predictor data set: an even
mix (even i: SBM, odd i: Chung-Lu) with N log-uniform in ``n_range`` and
k uniform in ``k_range``.
  * SBM: N rounded down to a multiple of k, mean degree s uniform in [8, 32],
    eps / eps_c uniform in [1/8, 1/2] (equal communities).
  * Chung-Lu: degree exponent uniform in [2.0, 3.0], mean degree uniform in
    [4, 12], largest expected degree sqrt(mean * N) (the weights' lower end is
    solved so the mean holds), every node of degree >= 1, connected; k is
    capped at N / 20 since these graphs have no planted communities.
``batched_sbm_set(seed)`` draws the block-diagonal batch: ``count`` SBMs with
N log-uniform in ``n_range``, k uniform in ``k_range``, N rounded to a
multiple of k (at least 10 k), mean degree 16 and eps = eps_c / 4; graph b
draws its size from its own generator, so graphs can be made in parallel.

Only input generation lives here (no arithmetic of the clustering method).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

from .graphs import CSRGraph, chung_lu, sbm


def _loguniform(rng: np.random.Generator, lo: float, hi: float) -> float:
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def bracket_graph(i: int, n_range: Tuple[float, float] = (1e4, 2e5),
                  k_range: Tuple[int, int] = (10, 500)) -> Tuple[CSRGraph, int]:
    """Graph i of the bracket data set and its k."""
    rng = np.random.Generator(np.random.PCG64(0x42524B54 + 7919 * i))
    n = int(round(_loguniform(rng, *n_range)))
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    if i % 2 == 0:
        k = max(2, min(k, n // 20))
        n = max(k * 20, (n // k) * k)
        s = float(rng.uniform(8.0, 32.0))
        ratio = float(rng.uniform(1.0 / 8.0, 1.0 / 2.0))
        g = sbm(n, k, s=s, seed=i, eps_over_epsc=ratio)
        g.meta.update(family="sbm", s=s, eps_over_epsc=ratio)
    else:
        exponent = float(rng.uniform(2.0, 3.0))
        mean = float(rng.uniform(4.0, 12.0))
        k = max(2, min(k, n // 20))
        g = chung_lu(n, exponent=exponent, mean=mean, seed=i, cutoff=math.sqrt(mean * n))
        g.meta.update(family="chung_lu")
    return g, k


def batched_sbm_graph(seed: int, b: int, n_range: Tuple[float, float] = (2e3, 5e4),
                      k_range: Tuple[int, int] = (5, 50)) -> Tuple[CSRGraph, int]:
    """Graph b of the block-diagonal batch drawn with ``seed``, and its k."""
    rng = np.random.Generator(np.random.PCG64(0x42415443 + 1000003 * seed + b))
    n = int(round(_loguniform(rng, *n_range)))
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    n = max(k * 10, (n // k) * k)
    return sbm(n, k, s=16.0, seed=seed * 100003 + b), k


def batched_sbm_set(seed: int = 0, count: int = 256, n_range: Tuple[float, float] = (2e3, 5e4),
                    k_range: Tuple[int, int] = (5, 50)) -> List[Tuple[CSRGraph, int]]:
    """``count`` SBM graphs of uneven size with their k (the block-diagonal batch)."""
    return [batched_sbm_graph(seed, b, n_range, k_range) for b in range(count)]


def batched_sbm_arrays(args):
    """Process-pool task: (seed, b) -> (b, row_ptr, col_idx, labels, k)."""
    seed, b = args
    g, k = batched_sbm_graph(seed, b)
    return b, g.row_ptr, g.col_idx, g.labels, k


def sizes_of(graphs: Sequence[Tuple[CSRGraph, int]]) -> np.ndarray:
    return np.array([g.n for g, _ in graphs], dtype=np.int64)


def bracket_graph_arrays(args):
    """Process-pool task: (i, n_range, k_range) -> (i, row_ptr, col_idx, labels, k)."""
    i, n_range, k_range = args
    g, k = bracket_graph(i, n_range, k_range)
    return i, g.row_ptr, g.col_idx, g.labels, k
