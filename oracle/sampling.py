"""Uniform sampling without replacement (Sec. 3.2 "Sampling and interpolation", Eq. 4)
and variable-density sampling (Sec. 3.2.3 after Theorem 3.4; remark closing Sec. 4.2).

Test infrastructure only.  The paper draws n indices Omega uniformly at
random from {1..N} without replacement and defines M_ij = 1 iff j = omega_i.
Reading (integer only, so both sides agree bit for bit): node i gets the key
k_i = output i of SplitMix64 seeded with ``seed``; Omega is the n nodes with
the smallest (k_i, i) in lexicographic order, returned sorted by node id.
Since the keys are i.i.d. uniform 64-bit words, every n-subset is equally
likely (ties between keys are broken by index and have probability ~2^-64).

Pins (tests/test_oracle_misc.py): exactly n distinct sorted indices;
inclusion frequency n/N per node over many seeds (chi-square); n = N returns
every node; the sampling matrix of Eq. 4 has one 1 per row.

Variable density.  The paper states that a sampling distribution shaped by
the local cumulative coherence v_k(i) = ||U_k^T delta_i|| needs only
O(k log k) samples whatever the graph, and that v_k(i) is estimated by the
row norm ||(H R)^T delta_i|| of the filtered signals (the quantity Alg. 2
step 4 divides by).  Readings, shared with the CUDA path:

* score s_i = ||(H~ R)^T delta_i||^2 of the UNnormalised filtered block (R
  has N(0, 1/d) entries, so E s_i = ||H~ delta_i||^2, which is v_k(i)^2 for
  the ideal low-pass); the distribution is p_i = s_i / sum_j s_j, the
  optimal density v_k(i)^2 / k of the cited sampling theory with the
  estimate in place of v_k(i);
* n draws i.i.d. WITH replacement (the cited theory's model), as an exact
  integer inverse CDF so that both sides choose the same nodes: weights
  q_i = floor(2^32 * (s_i / max_j s_j)) (one correctly rounded fp64
  division, an exact power-of-two scaling, floor), Q = sum q_i, draw t uses
  the word r_t = output t of SplitMix64 seeded with ``seed``, the point
  u_t = floor(r_t * Q / 2^64) (exact 128-bit product), and the node
  omega_t = the smallest i with q_0 + ... + q_i > u_t, so node i is drawn
  with probability q_i / Q up to 2^-64 per node; Omega is returned sorted,
  repeats adjacent;
* decoder weight of a draw of node i: w_i = Q / (N q_i) in fp64 (the
  P^{-1/2} weighting of the cited decoder, divided by N so that a uniform
  profile gives exactly w = 1 and gamma keeps its meaning), rounded to fp32.

Pins (tests/test_oracle_sampling.py): the inverse CDF against an exact
big-integer count of the 64-bit words mapped to each node; draw frequencies
against q (chi-square); a flat profile gives uniform draws and w = 1; zero
scores are never drawn; power-of-two rescaling changes nothing; the score
estimates ||H~ delta_i||^2 from an eigendecomposition (law of large numbers
in d).
"""
from __future__ import annotations

import numpy as np

from .rng import splitmix64_at

Q_BITS = 32


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


# --- variable-density sampling ------------------------------------------------

def coherence_scores(y: np.ndarray) -> np.ndarray:
    """s_i = ||(H~ R)^T delta_i||^2 of the unnormalised filtered block (fp64)."""
    y = np.asarray(y, dtype=np.float64)
    return np.einsum("ij,ij->i", y, y)


def quantize_scores(scores: np.ndarray) -> np.ndarray:
    """q_i = floor(2^32 * (s_i / max s)) as uint64; scores must be finite, >= 0, not all 0."""
    s = np.asarray(scores, dtype=np.float64)
    if s.ndim != 1 or len(s) == 0 or not np.all(np.isfinite(s)) or np.any(s < 0):
        raise ValueError("scores must be a non-empty vector of finite non-negative values")
    smax = float(s.max())
    if not smax > 0:
        raise ValueError("at least one score must be positive")
    return np.floor(np.ldexp(s / smax, Q_BITS)).astype(np.uint64)


def node_of_word(words: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Inverse CDF: u = floor(r * Q / 2^64), node = smallest i with q_0 + ... + q_i > u."""
    q = np.asarray(q, dtype=np.uint64)
    big_q = int(q.sum(dtype=np.uint64))
    cum = np.cumsum(q, dtype=np.uint64)
    u = np.array([(int(r) * big_q) >> 64 for r in np.asarray(words, dtype=np.uint64)], dtype=np.uint64)
    return np.searchsorted(cum, u, side="right").astype(np.int64)


def decoder_weights(q: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """w = Q / (N q_omega) in fp64, rounded to fp32."""
    q = np.asarray(q, dtype=np.uint64)
    big_q = np.float64(int(q.sum(dtype=np.uint64)))
    qo = q[np.asarray(omega, dtype=np.int64)].astype(np.float64)
    return (big_q / (np.float64(len(q)) * qo)).astype(np.float32)


def sample_variable_density(scores: np.ndarray, n: int, seed: int):
    """(Omega int64[n] sorted with repeats, decoder weights float32[n])."""
    if n < 0:
        raise ValueError("need n >= 0")
    q = quantize_scores(scores)
    omega = np.sort(node_of_word(splitmix64_at(seed, np.arange(n, dtype=np.uint64)), q))
    return omega, decoder_weights(q, omega)
