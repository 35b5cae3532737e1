"""A CPU model of the rounding that reduced-precision signal storage adds to the filter.

Test infrastructure: it derives the tolerance of the parity tests where the
pass band of h~ is a tiny share of the spectrum, so that the filtered block is
much smaller than the signals it is made from and storing the recurrence's
blocks in FP32 or BF16 loses more than the 1e-5 target on the normalised
features.  It is not the oracle (oracle/ holds the FP64 definition of the
method); it is a numpy restatement of the same Clenshaw evaluation
Y = sum_j c_j T_j(L - I) R (Clenshaw 1955; Sec. 2.1 "Fast graph filtering"), in
the pre-scaled form Z = D^-1/2 X whose neighbour sums are unweighted, with every
stored block (s R and each B_j) rounded to the storage type and the arithmetic
done in FP32:

  B_m = c_m s R,   B_j = c_j s R - 2 D^-1 W B_{j+1} - B_{j+2}   (j = m-1 .. 1),
  Y = D^1/2 (c_0 s R - D^-1 W B_1 - B_2),   s = D^-1/2 (1 for an isolated node).

Its summation order inside a neighbour sum is scipy's, not the kernels', so it
predicts the size of the storage error, not its bits.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (nearest, ties to even) and widen back to FP32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _store(x: np.ndarray, storage: str) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32)
    if storage == "f32":
        return x
    if storage == "bf16":
        return round_bf16(x)
    raise ValueError(f"unknown storage {storage!r}")


def clenshaw_stored(row_ptr: np.ndarray, col_idx: np.ndarray, r: np.ndarray, coeffs: np.ndarray,
                    storage: str = "f32") -> np.ndarray:
    """Y = h~(L) R with the stored blocks rounded to `storage` and FP32 arithmetic (see the module
    docstring); returns FP64 for comparison."""
    n = len(row_ptr) - 1
    deg = np.diff(np.asarray(row_ptr, dtype=np.int64)).astype(np.float64)
    w = sp.csr_matrix((np.ones(len(col_idx), np.float32), np.asarray(col_idx), np.asarray(row_ptr)), shape=(n, n))
    iso = deg == 0
    s = np.where(iso, 1.0, 1.0 / np.sqrt(np.where(iso, 1.0, deg))).astype(np.float32)[:, None]
    invdeg = np.where(iso, 0.0, 1.0 / np.where(iso, 1.0, deg)).astype(np.float32)[:, None]
    sqdeg = np.where(iso, 1.0, np.sqrt(deg)).astype(np.float32)[:, None]
    c = np.asarray(coeffs, dtype=np.float64).astype(np.float32)
    m = len(c) - 1
    sr = _store(s * np.asarray(r, dtype=np.float32), storage)
    if m == 0:
        return (sqdeg * (c[0] * sr)).astype(np.float64)
    two = np.float32(2.0)
    b2 = np.zeros_like(sr)
    b1 = _store(c[m] * sr, storage)
    for j in range(m - 1, 0, -1):
        bj = _store(c[j] * sr - two * invdeg * (w @ b1) - b2, storage)
        b2, b1 = b1, bj
    return (sqdeg * (c[0] * sr - invdeg * (w @ b1) - b2)).astype(np.float64)
