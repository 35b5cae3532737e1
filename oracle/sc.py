"""Spectral clustering, Alg. 1 (Ng, Jordan and Weiss's method on the normalized
Laplacian, Sec. 2.2), dense, for small graphs.  Test infrastructure only: the
comparison baseline of the recovery sweeps (Sec. 5.2, Fig. 1 a-d and f at
N = 1e3), not a product path.

Steps in the paper's order: the first k eigenvectors U_k of L (LAPACK eigh on
the dense Laplacian; ties inside a degenerate eigenspace give some orthonormal
basis of it, which the row normalisation and k-means do not depend on up to a
rotation), rows of U_k normalised to unit length (a zero row stays zero),
k-means on the N rows with the oracle's k-means (20 replicates, as the paper's
Matlab runs).  ``spectrum`` also returns the eigenvalues, the truth for the
lambda_k estimates of Fig. 1 e.

Pins (tests/test_oracle_sc.py): disjoint cliques and an SBM with eps = 0 are
recovered exactly; the span of U_k agrees with ARPACK's (scipy eigsh) through
the principal angles; on a two-community SBM the sign pattern of the Fiedler
vector of L (second eigenvector) gives the same partition.
"""
from __future__ import annotations

import numpy as np

from . import kmeans, laplacian


def spectrum(row_ptr, col_idx):
    """(eigenvalues ascending, eigenvectors as columns) of the dense normalized Laplacian."""
    return np.linalg.eigh(laplacian.dense_laplacian(row_ptr, col_idx))


def features(u_k: np.ndarray) -> np.ndarray:
    """Alg. 1 steps 2-3: rows of U_k scaled to unit length."""
    nrm = np.linalg.norm(u_k, axis=1, keepdims=True)
    return np.where(nrm > 0, u_k / np.where(nrm > 0, nrm, 1.0), 0.0)


def spectral_clustering(row_ptr, col_idx, k: int, seed: int = 0, replicates: int = 20, max_iter: int = 100):
    """Alg. 1: returns (labels int32[N], eigenvalues)."""
    ev, u = spectrum(row_ptr, col_idx)
    lab, _, _, _ = kmeans.kmeans(features(u[:, :k]), k, replicates, max_iter, seed)
    return np.asarray(lab, dtype=np.int32), ev
