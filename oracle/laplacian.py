"""Normalized Laplacian of Sec. 2.1 (test infrastructure only).

L = I - D^-1/2 W D^-1/2 with D_ii = sum_{j != i} W_ij.  The graphs are
unweighted (W_ij in {0, 1}), so the degree is the count of off-diagonal
entries of row i.  Reading for an isolated node (D_ii = 0, which the paper
excludes by assuming v_k(i) > 0): D^-1/2 is taken as 0 there, so the node is
an eigenvector of L with eigenvalue 1.

Pins: textbook spectra (k disjoint cliques, cycle, complete, complete
bipartite, path) and the bound 0 = lambda_1 <= ... <= lambda_N <= 2 of Sec. 2.1,
checked against LAPACK's dense eigensolver in tests/test_oracle_laplacian.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def adjacency(row_ptr: np.ndarray, col_idx: np.ndarray, weights=None) -> sp.csr_matrix:
    """W as a float64 CSR matrix with the diagonal (self loops) removed."""
    n = len(row_ptr) - 1
    data = np.ones(len(col_idx)) if weights is None else np.asarray(weights, dtype=np.float64)
    w = sp.csr_matrix((data, np.asarray(col_idx, dtype=np.int64), np.asarray(row_ptr, dtype=np.int64)),
                      shape=(n, n))
    w = w.tolil()
    w.setdiag(0.0)
    w = w.tocsr()
    w.eliminate_zeros()
    return w


def degrees(row_ptr: np.ndarray, col_idx: np.ndarray, weights=None) -> np.ndarray:
    """D_ii = sum_{j != i} W_ij (Sec. 2.1)."""
    return np.asarray(adjacency(row_ptr, col_idx, weights).sum(axis=1)).ravel()


def inv_sqrt_degrees(deg: np.ndarray) -> np.ndarray:
    out = np.zeros_like(deg, dtype=np.float64)
    pos = deg > 0
    out[pos] = 1.0 / np.sqrt(deg[pos])
    return out


def normalized_adjacency(row_ptr, col_idx, weights=None) -> sp.csr_matrix:
    """S = D^-1/2 W D^-1/2, so that L = I - S and L - I = -S."""
    w = adjacency(row_ptr, col_idx, weights)
    dinv = inv_sqrt_degrees(np.asarray(w.sum(axis=1)).ravel())
    dm = sp.diags(dinv)
    return (dm @ w @ dm).tocsr()


def laplacian(row_ptr, col_idx, weights=None) -> sp.csr_matrix:
    """L = I - D^-1/2 W D^-1/2 (Sec. 2.1)."""
    s = normalized_adjacency(row_ptr, col_idx, weights)
    n = s.shape[0]
    return (sp.identity(n, format="csr") - s).tocsr()


def dense_laplacian(row_ptr, col_idx, weights=None) -> np.ndarray:
    return laplacian(row_ptr, col_idx, weights).toarray()
