"""Seeded signal blocks and the workload definitions used by tests and bench.

``gaussian_block`` draws an N x d block of i.i.d. N(0, sigma^2) values (Alg. 2
step 3 uses sigma^2 = 1/d) with numpy's PCG64, laid out row-major with
``d_pad`` columns whose padding columns are zero.  The same array is handed
to the CUDA path and to the oracle, so a filter comparison isolates filter
error from generator error.

``score_profile`` draws a seeded vector of non-negative sampling scores (the
input of variable-density sampling) with one of a few shapes: heavy-tailed,
with runs of zeros, flat, a single positive entry, per-community constants.

``workload_sizes`` lists the parameter values of the five workloads (the
defaults of Alg. 2 with natural logarithms and ceilings).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_block(n: int, d: int, d_pad: int | None = None, seed: int = 0,
                   sigma: float | None = None, dtype=np.float32) -> np.ndarray:
    d_pad = d if d_pad is None else d_pad
    if d_pad < d:
        raise ValueError("d_pad < d")
    if sigma is None:
        sigma = 1.0 / math.sqrt(d) if d > 0 else 1.0
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((n, d_pad), dtype=np.float64)
    if d:
        out[:, :d] = rng.standard_normal((n, d)) * sigma
    return out.astype(dtype)


def score_profile(n: int, kind: str = "heavy", seed: int = 0) -> np.ndarray:
    """float64[n] of scores >= 0 with at least one positive entry."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "heavy":      # lognormal spread over ~8 decades
        out = np.exp(rng.normal(0.0, 4.0, n))
    elif kind == "zeros":    # about half exactly zero, the rest exponential
        out = rng.exponential(1.0, n) * (rng.random(n) < 0.5)
        out[rng.integers(0, n)] = 1.0
    elif kind == "flat":
        out = np.full(n, 0.37)
    elif kind == "single":
        out = np.zeros(n)
        out[rng.integers(0, n)] = 2.5
    elif kind == "blocks":   # constant within contiguous blocks of random sizes, 1 / size
        out = np.empty(n)
        i = 0
        while i < n:
            b = int(rng.integers(1, max(2, n // 8) + 1))
            out[i:i + b] = 1.0 / b
            i += b
    elif kind == "tiny":     # subnormal and normal values side by side
        out = rng.random(n) * 1e-300
        out[rng.integers(0, n)] = 5e-324
    else:
        raise ValueError(f"unknown score profile {kind!r}")
    return out.astype(np.float64)


def pad8(x: int) -> int:
    return ((x + 7) // 8) * 8


def workload_sizes(n_nodes: int, k: int) -> dict:
    """Alg. 2 defaults as read for the workloads: d = ceil(4 ln N), n = ceil(2k ln k),
    eigencount probes n_v = ceil(2 ln N), columns padded to a multiple of 8."""
    d = max(1, math.ceil(4 * math.log(n_nodes))) if n_nodes > 1 else 1
    n = min(n_nodes, max(k, math.ceil(2 * k * math.log(k)))) if k > 1 else min(n_nodes, 1)
    nv = max(1, math.ceil(2 * math.log(n_nodes))) if n_nodes > 1 else 1
    return dict(d=d, d_pad=pad8(d), n=n, n_v=nv, n_v_pad=pad8(nv))


# Named workloads (sizes only; graphs come from graphs.py with the given seed)
WORKLOADS = {
    "sbm_n1e3_k20": dict(kind="sbm", n=1000, k=20, s=16.0, m=50, gamma=1e-3, g_power=4, seed=0),
    "sbm_n1e5_k200": dict(kind="sbm", n=100_000, k=200, s=16.0, m=50, gamma=1e-3, g_power=4, seed=0),
    "chung_lu_n1e6_k100": dict(kind="chung_lu", n=1_000_000, k=100, exponent=2.1, mean=6.0,
                               m=100, gamma=1e-3, g_power=4, seed=0),
}
