"""Label interpolation of Eq. 5 and the partition rule of Sec. 4.1 (test infrastructure only).

Eq. 5: x_j = argmin ||M x - c_j^r||^2 + gamma x^T g(L) x, whose minimiser
solves (M^T M + gamma g(L)) x = M^T c_j^r, one system per cluster j
(Alg. 2 step 7).  M^T M is the diagonal 0/1 mask of sampled nodes.

Readings: g(L) = L^p with p = 4 and gamma = 1e-3 for the workloads (the
paper's preferred high-pass g = 1 - h~ is a separate option); the systems
are solved by conjugate gradients, one of the solvers Sec. 4.4 names, with
a diagonal preconditioner mask + gamma, to relative residual 1e-10.  On a
connected component holding no sample the right-hand side is zero and the
solution there is zero.  Labels: node i goes to the j maximising
x_j(i) / ||x_j|| (ties to the lowest j; a zero column scores 0).

Pins (tests/test_oracle_misc.py): agreement with a dense LAPACK solve;
n = N with gamma -> 0 returns c^r; on disjoint regular cliques with every
clique sampled the indicators lie in ker L, so x_j is the exact indicator.
Weighted decoder (variable-density draws, see the comment above
interpolate_weighted; tests/test_oracle_sampling.py): unit weights on distinct
draws reproduce Eq. 5; a node drawn twice equals one draw of twice the
weight; the solution is a stationary point of the objective written term by
term over the draws (finite differences) and beats random perturbations.
High-pass variant: agreement with the system built from LAPACK eigh
(g~(L) = U (1 - h~(Lambda)) U^T); on disjoint cliques the indicators lie in the
pass band (h~ = 1 up to the Jackson error at lambda = 0), so x_j is within that
error of the indicator.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def rhs(n_nodes: int, omega: np.ndarray, sample_labels: np.ndarray, k: int) -> np.ndarray:
    """B = M^T C^r: column j holds 1 at sampled nodes labelled j."""
    b = np.zeros((n_nodes, k))
    b[np.asarray(omega, dtype=np.int64), np.asarray(sample_labels, dtype=np.int64)] = 1.0
    return b


def mask(n_nodes: int, omega: np.ndarray) -> np.ndarray:
    m = np.zeros(n_nodes)
    m[np.asarray(omega, dtype=np.int64)] = 1.0
    return m


def system_matrix(lap: sp.csr_matrix, msk: np.ndarray, gamma: float, power: int) -> sp.csr_matrix:
    """M^T M + gamma L^p as an explicit sparse matrix (small graphs)."""
    g = sp.identity(lap.shape[0], format="csr")
    for _ in range(power):
        g = g @ lap
    return (sp.diags(msk) + gamma * g).tocsr()


def apply_system(lap: sp.csr_matrix, msk: np.ndarray, gamma: float, power: int, x: np.ndarray) -> np.ndarray:
    """(M^T M + gamma L^p) x with p successive products by L."""
    t = x
    for _ in range(power):
        t = lap @ t
    return msk[:, None] * x + gamma * t if x.ndim == 2 else msk * x + gamma * t


def cg(apply, b: np.ndarray, precond: np.ndarray, tol: float = 1e-10, max_iter: int = 20000):
    """Preconditioned CG on every column of b independently.

    Returns (x, iterations, max relative residual).
    """
    x = np.zeros_like(b)
    r = b.copy()
    z = r / precond[:, None]
    p = z.copy()
    rz = np.sum(r * z, axis=0)
    bn = np.linalg.norm(b, axis=0)
    active = bn > 0
    it = 0
    for it in range(1, max_iter + 1):
        rn = np.linalg.norm(r, axis=0)
        conv = ~active | (rn <= tol * np.where(bn > 0, bn, 1.0))
        if np.all(conv):
            it -= 1
            break
        ap = apply(p)
        pap = np.sum(p * ap, axis=0)
        alpha = np.where(conv | (pap == 0), 0.0, rz / np.where(pap == 0, 1.0, pap))
        x += alpha * p
        r -= alpha * ap
        z = r / precond[:, None]
        rz_new = np.sum(r * z, axis=0)
        beta = np.where(conv | (rz == 0), 0.0, rz_new / np.where(rz == 0, 1.0, rz))
        p = np.where(conv, p, z + beta * p)
        rz = np.where(conv, rz, rz_new)
    rel = np.linalg.norm(b - apply(x), axis=0) / np.where(bn > 0, bn, 1.0)
    return x, it, float(np.max(rel)) if rel.size else 0.0


def interpolate(lap: sp.csr_matrix, omega: np.ndarray, sample_labels: np.ndarray, k: int,
                gamma: float = 1e-3, power: int = 4, tol: float = 1e-10, max_iter: int = 20000):
    """Solve Eq. 5 for every cluster; returns (X int N x k, iterations, max rel residual)."""
    n_nodes = lap.shape[0]
    msk = mask(n_nodes, omega)
    b = rhs(n_nodes, omega, sample_labels, k)
    pre = msk + gamma
    x, it, res = cg(lambda v: apply_system(lap, msk, gamma, power, v), b, pre, tol, max_iter)
    return x, it, res


# --- the paper's high-pass choice: g = 1 - h~_{lambda_k} (Sec. 4.4 after Eq. 5) ---
# g~(L) = I - h~(L), h~ the Jackson-Chebyshev low-pass of degree m at the cut-off
# lambda_k (the filter of Alg. 2 step 4), applied with the forward recurrence.

def apply_highpass(s_mat: sp.csr_matrix, msk: np.ndarray, gamma: float, lam: float, m: int,
                   x: np.ndarray) -> np.ndarray:
    """(M^T M + gamma (I - h~(L))) x, with h~(L) x by the oracle's Chebyshev filter."""
    from . import chebyshev as och

    xx = x if x.ndim == 2 else x[:, None]
    hx = och.cheb_filter(s_mat, xx, och.filter_coeffs(lam, m))
    out = msk[:, None] * xx + gamma * (xx - hx)
    return out if x.ndim == 2 else out[:, 0]


def interpolate_highpass(s_mat: sp.csr_matrix, omega: np.ndarray, sample_labels: np.ndarray, k: int,
                         lam: float, m: int, gamma: float = 1e-3, tol: float = 1e-10, max_iter: int = 20000):
    """Eq. 5 with g = 1 - h~_{lambda}: (X, iterations, max rel residual); s_mat = D^-1/2 W D^-1/2."""
    n_nodes = s_mat.shape[0]
    msk = mask(n_nodes, omega)
    b = rhs(n_nodes, omega, sample_labels, k)
    pre = msk + gamma
    return cg(lambda v: apply_highpass(s_mat, msk, gamma, lam, m, v), b, pre, tol, max_iter)


def interpolate_highpass_dense(lap_dense: np.ndarray, omega, sample_labels, k, lam, m, gamma=1e-3):
    """The same system built from the eigendecomposition: g~(L) = U (1 - h~(Lambda)) U^T."""
    from . import chebyshev as och

    n_nodes = lap_dense.shape[0]
    w, u = np.linalg.eigh(lap_dense)
    g = u @ np.diag(1.0 - och.h_tilde(w, lam, m)) @ u.T
    a = np.diag(mask(n_nodes, omega)) + gamma * g
    return np.linalg.solve(a, rhs(n_nodes, omega, sample_labels, k))


def interpolate_dense(lap_dense: np.ndarray, omega, sample_labels, k, gamma=1e-3, power=4):
    n_nodes = lap_dense.shape[0]
    a = np.diag(mask(n_nodes, omega)) + gamma * np.linalg.matrix_power(lap_dense, power)
    return np.linalg.solve(a, rhs(n_nodes, omega, sample_labels, k))


# --- weighted decoder for variable-density samples -----------------------------
# The sampling theory the paper cites for variable density (Sec. 3.2.3 after
# Theorem 3.4) decodes with the fidelity term weighted by P^{-1/2}:
#   x_j = argmin_x sum_t w_t (x(omega_t) - c_j(t))^2 + gamma x^T g(L) x,
# the sum over draws t (a node drawn twice counts twice), w_t = 1 / (N p_t).
# Normal equations: (M^T W M + gamma g(L)) x = M^T W c_j; M^T W M is diagonal
# with the summed weights of each node's draws.  Unit weights and distinct
# draws give Eq. 5 exactly.

def weighted_mask(n_nodes: int, omega: np.ndarray, w: np.ndarray) -> np.ndarray:
    m = np.zeros(n_nodes)
    np.add.at(m, np.asarray(omega, dtype=np.int64), np.asarray(w, dtype=np.float64))
    return m


def weighted_rhs(n_nodes: int, omega: np.ndarray, sample_labels: np.ndarray, w: np.ndarray, k: int) -> np.ndarray:
    b = np.zeros((n_nodes, k))
    np.add.at(b, (np.asarray(omega, dtype=np.int64), np.asarray(sample_labels, dtype=np.int64)),
              np.asarray(w, dtype=np.float64))
    return b


def interpolate_weighted(lap: sp.csr_matrix, omega: np.ndarray, sample_labels: np.ndarray, w: np.ndarray, k: int,
                         gamma: float = 1e-3, power: int = 4, tol: float = 1e-10, max_iter: int = 20000):
    """Weighted Eq. 5 for every cluster; returns (X, iterations, max rel residual)."""
    n_nodes = lap.shape[0]
    msk = weighted_mask(n_nodes, omega, w)
    b = weighted_rhs(n_nodes, omega, sample_labels, w, k)
    return cg(lambda v: apply_system(lap, msk, gamma, power, v), b, msk + gamma, tol, max_iter)


def weighted_objective(lap_dense: np.ndarray, omega, sample_labels, w, gamma: float, power: int,
                       x: np.ndarray) -> np.ndarray:
    """The weighted objective of every column of x, term by term over the draws (small cases)."""
    k = x.shape[1]
    g = np.linalg.matrix_power(lap_dense, power)
    out = np.zeros(k)
    for j in range(k):
        for t in range(len(omega)):
            target = 1.0 if sample_labels[t] == j else 0.0
            out[j] += float(w[t]) * (x[omega[t], j] - target) ** 2
        out[j] += gamma * x[:, j] @ g @ x[:, j]
    return out


def labels_from_indicators(x: np.ndarray) -> np.ndarray:
    """Sec. 4.1: node i -> argmax_j x_j(i) / ||x_j|| (ties to the lowest j)."""
    nrm = np.linalg.norm(x, axis=0)
    scaled = np.where(nrm > 0, x / np.where(nrm > 0, nrm, 1.0), 0.0)
    return np.argmax(scaled, axis=1).astype(np.int32)
