"""Features and targets of the learned lambda_k bracket (test infrastructure only).

The paper estimates lambda_k by a dichotomy on an eigencount (Sec. 4.3) and is
silent on learning it.  The learned predictor maps cheap graph statistics to
an interval that should contain an acceptable dichotomy answer; the eigencount
still decides whether that interval holds one.  Readings:

* Features (72 values):
    0..63   mu_j / N, j = 0..63: eigencount moments (Sec. 4.3 estimator) of
            8 N(0, 1) probes (the first 8 probe columns of the shared Philox
            convention), by the direct recurrence;
    64      ln N;
    65      k;
    66..71  ln(1 + q) for the degree quantiles q at 0, 0.1, 0.25, 0.5, 0.75, 1,
            where the quantile at p is the sorted degree at index floor(p (N - 1)).
* Target bracket [lambda_lo, lambda_hi]: the cut-offs where count(lambda), from
  moments of degree m with the full probe count, equals k - 1/2 and k + 1/2.
  Every lambda inside rounds to count k, i.e. is an answer the dichotomy of
  Sec. 4.3 accepts.  count is nondecreasing in lambda (the damped step moves
  its transition to the right as lambda grows and the Jackson kernel is
  nonnegative), so each crossing is found by bisection on [0, 2] (60 halvings).
* Regression target: (centre, ln half-width) of that bracket.

Pins (tests/test_oracle_mlp.py): the quantile rule equals numpy's
``quantile(method="lower")``; on disjoint cliques with every basis vector as a
probe the count is exact, so the bracket lies inside the spectral gap
(0, s/(s-1)); crossing values are met to 1e-9.
"""
from __future__ import annotations

import math

import numpy as np

from . import chebyshev as och
from . import laplacian as olap

FEATURE_PROBES = 8
FEATURE_MOMENTS = 64
QUANTILES = (0.0, 0.1, 0.25, 0.5, 0.75, 1.0)
N_FEATURES = FEATURE_MOMENTS + 2 + len(QUANTILES)


def degree_quantiles(deg: np.ndarray) -> np.ndarray:
    d = np.sort(np.asarray(deg, dtype=np.int64))
    n = d.size
    return np.array([d[int(math.floor(p * (n - 1)))] for p in QUANTILES], dtype=np.float64)


def features_from(mu64: np.ndarray, n: int, k: int, deg: np.ndarray) -> np.ndarray:
    f = np.empty(N_FEATURES, dtype=np.float64)
    f[:FEATURE_MOMENTS] = np.asarray(mu64, dtype=np.float64)[:FEATURE_MOMENTS] / n
    f[FEATURE_MOMENTS] = math.log(n)
    f[FEATURE_MOMENTS + 1] = k
    f[FEATURE_MOMENTS + 2:] = np.log1p(degree_quantiles(deg))
    return f


def features(row_ptr: np.ndarray, col_idx: np.ndarray, k: int, seed: int) -> np.ndarray:
    """The 72 features of one graph (moments of 8 probes drawn with ``seed``)."""
    s = olap.normalized_adjacency(row_ptr, col_idx)
    n = s.shape[0]
    probes = och.probe_signals(n, FEATURE_PROBES, FEATURE_PROBES, seed)
    mu = och.moments(s, probes, FEATURE_MOMENTS - 1)
    return features_from(mu, n, k, olap.degrees(row_ptr, col_idx))


def crossing(mu: np.ndarray, level: float, iters: int = 60) -> float:
    """Smallest-bracket bisection for count(lambda) = level on [0, 2]."""
    lo, hi = 0.0, 2.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if och.eigencount(mu, mid) < level:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def target_bracket(mu: np.ndarray, k: int) -> tuple[float, float]:
    """[lambda_lo, lambda_hi] where count crosses k - 1/2 and k + 1/2."""
    return crossing(mu, k - 0.5), crossing(mu, k + 0.5)


def bracket_to_target(lo: float, hi: float) -> np.ndarray:
    return np.array([0.5 * (lo + hi), math.log(max(0.5 * (hi - lo), 1e-12))])


def target_to_bracket(t: np.ndarray, widen: float = 1.0) -> tuple[float, float]:
    """(centre, ln half-width) -> [lo, hi], half-width scaled by ``widen``, clipped to [0, 2]."""
    c, hw = float(t[0]), widen * math.exp(float(t[1]))
    return max(0.0, c - hw), min(2.0, c + hw)
