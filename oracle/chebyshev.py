"""Jackson-Chebyshev filtering and eigencount (test infrastructure only).

Follows, in FP64:

* Eq. 1 -- the ideal low-pass h_{lambda_c}(lambda) = 1 if lambda <= lambda_c else 0.
* Sec. 2.1 "Fast graph filtering" -- h(L) x is approximated by a polynomial in L
  applied with successive sparse products, never forming h(L).
* Sec. 4.3 "The polynomial approximation" -- Jackson-Chebyshev polynomials
  (Chebyshev expansion plus Jackson damping factors, after Di Napoli, Polizzi
  and Saad).  The spectrum of L lies in [0, 2] (Sec. 2.1), so the map to the
  Chebyshev interval is t = lambda - 1, i.e. the operator L - I = -S.
* Alg. 2 step 4 -- Y = h~(L) R and the row normalisation f_i = Y_i / ||Y_i||.
* Sec. 4.3 "Estimation of lambda_k" -- eigencount by low-pass filtering random
  probes and a dichotomy on lambda starting from lambda = 2.

Readings (the paper does not print these formulas):
* "order p" = polynomial degree m: terms j = 0..m.
* Chebyshev coefficients of the indicator of [-1, t_c] with theta_c = arccos(t_c):
  gamma_0 = 1 - theta_c / pi, gamma_j = -2 sin(j theta_c) / (j pi).
* Jackson damping, alpha = pi / (m + 2):
  g_j = [(1 - j/(m+2)) sin(alpha) cos(j alpha) + cos(alpha) sin(j alpha) / (m+2)] / sin(alpha).
* Eigencount estimator: count(lambda) = (1/n_v) sum_l r_l^T h~_lambda(L) r_l with
  N(0, 1) probes r_l, n_v = ceil(2 ln N); since h~_lambda(L) = sum_j c_j(lambda) T_j(L - I),
  count(lambda) = sum_j c_j(lambda) mu_j with moments mu_j = (1/n_v) sum_l r_l^T T_j(L - I) r_l.
* Dichotomy: lo = 0, hi = 2; at mid = (lo + hi)/2, stop if round(count) = k
  (round half away from zero); if count > k then hi = mid else lo = mid;
  give up after 60 halvings or when hi - lo < 1e-12 and return hi, flagged.

Pins (tests/test_oracle_chebyshev.py): g_0 = 1 and g_{m+1} = 0 exactly;
the damped filter stays within [0, 1] (Jackson kernel positivity); gamma_j
against Chebyshev-Gauss quadrature of the step; the filtered block against
U h~(Lambda) U^T R from LAPACK's dense eigensolver; ideal-filter limit
U_k U_k^T R at large m across a spectral gap; the eigencount with all N basis
vectors as probes equals sum_i h~(lambda_i) and, in a gap, #{lambda_i <= lambda};
count(0) = 0 on a graph whose spectrum starts above 0 ... see the tests.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import rng as _rng


def jackson_factor(m: int, j) -> np.ndarray:
    """Jackson damping factor g_j of the degree-m expansion (Sec. 4.3, after Di Napoli et al.)."""
    j = np.asarray(j, dtype=np.float64)
    a = math.pi / (m + 2)
    return ((1.0 - j / (m + 2)) * math.sin(a) * np.cos(j * a)
            + math.cos(a) * np.sin(j * a) / (m + 2)) / math.sin(a)


def jackson(m: int) -> np.ndarray:
    """Jackson damping factors g_0..g_m for degree m."""
    return jackson_factor(m, np.arange(m + 1))


def step_gamma(lambda_c: float, m: int) -> np.ndarray:
    """Chebyshev coefficients of the ideal low-pass of Eq. 1 on t = lambda - 1."""
    t_c = min(max(lambda_c - 1.0, -1.0), 1.0)
    th = math.acos(t_c)
    g = np.empty(m + 1, dtype=np.float64)
    g[0] = 1.0 - th / math.pi
    if m >= 1:
        j = np.arange(1, m + 1, dtype=np.float64)
        g[1:] = -2.0 * np.sin(j * th) / (j * math.pi)
    return g


def filter_coeffs(lambda_c: float, m: int, damped: bool = True) -> np.ndarray:
    """c_j = g_j gamma_j (damped) or gamma_j (truncated Chebyshev)."""
    c = step_gamma(lambda_c, m)
    return c * jackson(m) if damped else c


def chebyshev_T(j: int, t: np.ndarray) -> np.ndarray:
    """T_j(t) = cos(j arccos t) on [-1, 1]."""
    return np.cos(j * np.arccos(np.clip(t, -1.0, 1.0)))


def h_tilde(lam, lambda_c: float, m: int, damped: bool = True) -> np.ndarray:
    """The polynomial h~_{lambda_c}(lambda) = sum_j c_j T_j(lambda - 1)."""
    lam = np.asarray(lam, dtype=np.float64)
    c = filter_coeffs(lambda_c, m, damped)
    th = np.arccos(np.clip(lam - 1.0, -1.0, 1.0))
    j = np.arange(m + 1, dtype=np.float64)
    return np.cos(np.multiply.outer(th, j)) @ c


def cheb_filter(s: sp.csr_matrix, r: np.ndarray, coeffs: np.ndarray) -> np.ndarray:
    """Y = sum_j c_j T_j(L - I) R by the three-term recurrence (Sec. 2.1, Alg. 2 step 4).

    X_0 = R, X_1 = (L - I) R = -S R, X_{j+1} = 2 (L - I) X_j - X_{j-1}.
    """
    r = np.asarray(r, dtype=np.float64)
    m = len(coeffs) - 1
    x_prev = r
    y = coeffs[0] * x_prev
    if m == 0:
        return y
    x_cur = -(s @ x_prev)
    y = y + coeffs[1] * x_cur
    for j in range(1, m):
        x_next = -2.0 * (s @ x_cur) - x_prev
        y = y + coeffs[j + 1] * x_next
        x_prev, x_cur = x_cur, x_next
    return y


def normalize_rows(y: np.ndarray) -> np.ndarray:
    """f_i = Y_i / ||Y_i|| (Alg. 2 step 4); a zero row stays zero."""
    nrm = np.sqrt(np.sum(y * y, axis=1))
    out = np.zeros_like(y)
    pos = nrm > 0
    out[pos] = y[pos] / nrm[pos, None]
    return out


def random_signals(n: int, d: int, d_pad: int, seed: int) -> np.ndarray:
    """Alg. 2 step 3: N(0, 1/d) signals, by the shared Philox convention."""
    return _rng.gaussian_block(n, d, d_pad, seed, _rng.STREAM_SIGNALS, 1.0 / math.sqrt(max(d, 1)))


def probe_signals(n: int, n_v: int, n_v_pad: int, seed: int) -> np.ndarray:
    """Sec. 4.3 eigencount probes: N(0, 1) signals, by the shared Philox convention."""
    return _rng.gaussian_block(n, n_v, n_v_pad, seed, _rng.STREAM_PROBES, 1.0)


def moments(s: sp.csr_matrix, probes: np.ndarray, m: int, n_v: int | None = None) -> np.ndarray:
    """mu_j = (1/n_v) sum_l r_l^T T_j(L - I) r_l, j = 0..m, by the direct recurrence."""
    p = np.asarray(probes, dtype=np.float64)
    n_v = p.shape[1] if n_v is None else n_v
    mu = np.zeros(m + 1)
    x_prev = p
    mu[0] = np.sum(p * x_prev) / n_v
    if m == 0:
        return mu
    x_cur = -(s @ p)
    mu[1] = np.sum(p * x_cur) / n_v
    for j in range(1, m):
        x_next = -2.0 * (s @ x_cur) - x_prev
        mu[j + 1] = np.sum(p * x_next) / n_v
        x_prev, x_cur = x_cur, x_next
    return mu


def eigencount(mu: np.ndarray, lam: float, damped: bool = True) -> float:
    """count(lambda) = sum_j c_j(lambda) mu_j (Sec. 4.3 estimator, moments form)."""
    m = len(mu) - 1
    return float(np.dot(filter_coeffs(lam, m, damped), mu))


def eigencount_refilter(s: sp.csr_matrix, probes: np.ndarray, lam: float, m: int,
                        damped: bool = True, n_v: int | None = None) -> float:
    """The paper-literal estimator: filter the probes at cut-off lam, then average r^T h~(L) r."""
    p = np.asarray(probes, dtype=np.float64)
    n_v = p.shape[1] if n_v is None else n_v
    y = cheb_filter(s, p, filter_coeffs(lam, m, damped))
    return float(np.sum(p * y) / n_v)


def round_half_away(x: float) -> int:
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def dichotomy(count_fn, k: int, max_iter: int = 60, width_tol: float = 1e-12):
    """Sec. 4.3: halve [0, 2] until round(count(lambda)) = k.

    Returns (lambda, count(lambda), iterations, hit) where hit is False when
    the bracket collapsed without an exact hit (lambda = hi is returned).
    """
    lo, hi = 0.0, 2.0
    for it in range(1, max_iter + 1):
        mid = 0.5 * (lo + hi)
        c = count_fn(mid)
        if round_half_away(c) == k:
            return mid, c, it, True
        if c > k:
            hi = mid
        else:
            lo = mid
        if hi - lo < width_tol:
            return hi, count_fn(hi), it, False
    return hi, count_fn(hi), max_iter, False


def estimate_lambda_k(s: sp.csr_matrix, k: int, m: int, n_v: int, seed: int,
                      damped: bool = True):
    """Alg. 2 step 1 with moments computed once and every threshold evaluated from them."""
    n = s.shape[0]
    probes = probe_signals(n, n_v, n_v, seed)
    mu = moments(s, probes, m)
    lam, c, it, hit = dichotomy(lambda x: eigencount(mu, x, damped), k)
    return dict(lam=lam, count=c, iters=it, hit=hit, mu=mu)
