"""Alg. 2 (Compressive Spectral Clustering) end to end in FP64, test infrastructure only.

Steps, in the paper's order, each delegated to the module that follows it:
1. estimate lambda_k by eigencount and dichotomy (chebyshev, Sec. 4.3), with the
   eigencount filter of degree m_count (default m; the paper does not fix it);
2. Jackson-Chebyshev coefficients of h_{lambda_k} (chebyshev, Sec. 4.3);
3. R: d signals N(0, 1/d) (rng, shared Philox convention);
4. Y = h~(L) R, rows normalised (chebyshev, Alg. 2 step 4);
5. Omega: n nodes uniformly without replacement (sampling, Eq. 4), or n
   variable-density draws with scores ||Y_i||^2 of the unnormalised block
   (sampling, Sec. 3.2.3 and the remark closing Sec. 4.2);
6. k-means on the n sampled feature rows (kmeans);
7. interpolation by Eq. 5 (weighted by the draws' 1 / (N p) under variable
   density) and the argmax rule (interp, Sec. 4.1).

The paper prints no recovery value (its figures are absent), so on SBMs the
end-to-end results are checked against the planted communities and against
the CUDA path, not against a printed number.  Pinned where the answer is
fixed: on disjoint cliques (lambda_1..k = 0, an exact spectral gap) the
pipeline returns the cliques exactly (tests/test_oracle_misc.py).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import chebyshev, interp, kmeans, laplacian, sampling


def defaults(n_nodes: int, k: int) -> dict:
    """Parameter reading: d = ceil(4 ln N), n = ceil(2 k ln k), n_v = ceil(2 ln N), m = 50, gamma = 1e-3."""
    d = max(1, math.ceil(4 * math.log(n_nodes))) if n_nodes > 1 else 1
    n = min(n_nodes, max(k, math.ceil(2 * k * math.log(k)))) if k > 1 else min(n_nodes, 1)
    nv = max(1, math.ceil(2 * math.log(n_nodes))) if n_nodes > 1 else 1
    return dict(d=d, n=n, n_v=nv, m=50, gamma=1e-3, g_power=4)


def csc(row_ptr, col_idx, k: int, seed: int = 0, m: int = 50, d: int | None = None,
        n: int | None = None, n_v: int | None = None, gamma: float = 1e-3, g_power: int = 4,
        replicates: int = 20, max_iter_km: int = 100, cg_tol: float = 1e-10,
        lambda_k: float | None = None, r_in: np.ndarray | None = None, timings: dict | None = None,
        variable_density: bool = False, m_count: int | None = None):
    """Run Alg. 2 and return a dict with every intermediate result."""
    t0 = time.perf_counter()
    n_nodes = len(row_ptr) - 1
    dflt = defaults(n_nodes, k)
    d = dflt["d"] if d is None else d
    n = dflt["n"] if n is None else n
    n_v = dflt["n_v"] if n_v is None else n_v
    s = laplacian.normalized_adjacency(row_ptr, col_idx)
    lap = laplacian.laplacian(row_ptr, col_idx)
    tt = {}
    t = time.perf_counter()
    if lambda_k is None:
        est = chebyshev.estimate_lambda_k(s, k, m if m_count is None else m_count, n_v, seed)
        lam = est["lam"]
    else:
        est, lam = None, lambda_k
    tt["lambda_k"] = time.perf_counter() - t
    t = time.perf_counter()
    coeffs = chebyshev.filter_coeffs(lam, m)
    r = chebyshev.random_signals(n_nodes, d, d, seed) if r_in is None else np.asarray(r_in, np.float64)
    y = chebyshev.cheb_filter(s, r, coeffs)
    feats = chebyshev.normalize_rows(y)
    tt["filter"] = time.perf_counter() - t
    t = time.perf_counter()
    if variable_density:
        omega, w = sampling.sample_variable_density(sampling.coherence_scores(y), n, seed)
    else:
        omega, w = sampling.sample(n_nodes, n, seed), None
    lab_r, _, inertia, _ = kmeans.kmeans(feats[omega], k, replicates, max_iter_km, seed)
    tt["kmeans"] = time.perf_counter() - t
    t = time.perf_counter()
    if w is None:
        x, cg_it, cg_res = interp.interpolate(lap, omega, lab_r, k, gamma, g_power, cg_tol)
    else:
        x, cg_it, cg_res = interp.interpolate_weighted(lap, omega, lab_r, w, k, gamma, g_power, cg_tol)
    labels = interp.labels_from_indicators(x)
    tt["interp"] = time.perf_counter() - t
    tt["total"] = time.perf_counter() - t0
    if timings is not None:
        timings.update(tt)
    return dict(lam=lam, est=est, coeffs=coeffs, r=r, y=y, features=feats, omega=omega, weights=w,
                sample_labels=lab_r, inertia=inertia, x=x, cg_iters=cg_it, cg_res=cg_res,
                labels=labels, params=dict(k=k, m=m, m_count=m if m_count is None else m_count, d=d, n=n, n_v=n_v,
                                           gamma=gamma,
                                           g_power=g_power, seed=seed))
