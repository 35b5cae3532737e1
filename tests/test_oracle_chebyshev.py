"""Pins of the oracle's Jackson-Chebyshev filter and eigencount (Eq. 1, Sec. 2.1, Sec. 4.3)."""
import math

import numpy as np
import pytest

import csc_inputs as ci
from oracle import chebyshev as ch
from oracle import laplacian


@pytest.mark.parametrize("m", [0, 1, 2, 10, 50, 100])
def test_jackson_endpoints(m):
    g = ch.jackson(m)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert abs(float(ch.jackson_factor(m, m + 1))) < 1e-14
    assert np.all(np.diff(g) <= 1e-15)  # damping decreases with j
    assert np.all(g > 0)


@pytest.mark.parametrize("m", [5, 20, 50, 100])
@pytest.mark.parametrize("lam_c", [0.05, 0.3, 1.0, 1.7])
def test_damped_filter_in_unit_interval(m, lam_c):
    lam = np.linspace(0, 2, 100001)
    h = ch.h_tilde(lam, lam_c, m)
    assert h.min() > -1e-13 and h.max() < 1 + 1e-13
    # a positive kernel smoothing a longer step gives a larger value: h~ grows with
    # the cut-off at every fixed lambda, which is what makes the dichotomy monotone
    h2 = ch.h_tilde(lam, lam_c + 0.01, m)
    assert np.all(h2 - h > -1e-13)


@pytest.mark.parametrize("lam_c", [0.2, 0.9, 1.5])
def test_gamma_matches_gauss_chebyshev_quadrature(lam_c):
    m, q = 40, 1_000_000
    th = math.pi * (np.arange(q) + 0.5) / q
    f = (np.cos(th) <= lam_c - 1.0).astype(np.float64)
    quad = np.array([(2.0 if j else 1.0) / q * np.sum(f * np.cos(j * th)) for j in range(m + 1)])
    assert np.allclose(ch.step_gamma(lam_c, m), quad, atol=5e-6)


def test_truncated_chebyshev_converges_away_from_jump():
    lam_c = 0.7
    lam = np.array([0.1, 0.3, 1.1, 1.6])
    err = [np.max(np.abs(ch.h_tilde(lam, lam_c, m, damped=False) - (lam <= lam_c))) for m in (20, 80, 320)]
    assert err[2] < err[0]
    assert np.max(np.abs(ch.h_tilde(lam, lam_c, 400) - (lam <= lam_c))) < 1e-3


def test_recurrence_matches_chebyshev_polynomials():
    t = np.linspace(-1, 1, 7)
    s = np.diag(-t)  # so that L - I = -S = diag(t)
    import scipy.sparse as sp
    e = np.eye(7)
    for j in range(6):
        c = np.zeros(j + 1)
        c[j] = 1.0
        y = ch.cheb_filter(sp.csr_matrix(s), e, c)
        assert np.allclose(np.diag(y), ch.chebyshev_T(j, t), atol=1e-13)


def _dense(g):
    lap = laplacian.dense_laplacian(g.row_ptr, g.col_idx)
    w, u = np.linalg.eigh(lap)
    return lap, w, u


@pytest.mark.parametrize("m", [0, 1, 2, 7, 50])
def test_filter_matches_dense_spectral_definition(m):
    g = ci.sbm(240, 6, s=10, seed=5)
    lap, w, u = _dense(g)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    r = ci.gaussian_block(240, 9, 9, seed=2, dtype=np.float64)
    lam_c = 0.45
    y = ch.cheb_filter(s, r, ch.filter_coeffs(lam_c, m))
    ref = u @ (ch.h_tilde(w, lam_c, m)[:, None] * (u.T @ r))
    assert np.linalg.norm(y - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300) + 1e-13


def test_filter_approaches_ideal_projection_across_gap():
    # 5 cliques of 20 joined by a few edges: lambda_5 small, lambda_6 near 20/19
    base = ci.disjoint_cliques(5, 20)
    i, j = base.edges()
    extra_i = np.array([0, 20, 40, 60, 80])
    extra_j = np.array([25, 45, 65, 85, 5])
    g = ci.from_edges(100, np.concatenate([i, extra_i]), np.concatenate([j, extra_j]))
    lap, w, u = _dense(g)
    assert w[4] < 0.2 and w[5] > 0.9
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    r = ci.gaussian_block(100, 6, 6, seed=1, dtype=np.float64)
    y = ch.cheb_filter(s, r, ch.filter_coeffs(0.5, 400))
    uk = u[:, :5]
    ref = uk @ (uk.T @ r)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-6


def test_eigencount_with_basis_probes_is_trace():
    g = ci.sbm(150, 5, s=8, seed=9)
    lap, w, u = _dense(g)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    n = 150
    probes = math.sqrt(n) * np.eye(n)
    m = 60
    mu = ch.moments(s, probes, m)
    for lam in (0.1, 0.4, 0.8, 1.3, 2.0):
        exact = float(np.sum(ch.h_tilde(w, lam, m)))
        assert ch.eigencount(mu, lam) == pytest.approx(exact, rel=1e-12, abs=1e-10)


def test_eigencount_in_gap_counts_eigenvalues():
    g = ci.disjoint_cliques(7, 12)
    lap, w, u = _dense(g)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    n = g.n
    mu = ch.moments(s, math.sqrt(n) * np.eye(n), 120)
    # spectrum: 0 (x7) and 12/11 (x77); lambda = 0.5 sits in the gap
    assert ch.round_half_away(ch.eigencount(mu, 0.5)) == 7
    assert ch.round_half_away(ch.eigencount(mu, 1.6)) == n


def test_eigencount_endpoints():
    g = ci.sbm(120, 4, s=8, seed=1)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    p = ch.probe_signals(120, 8, 8, seed=3)
    mu = ch.moments(s, p, 50)
    assert abs(ch.eigencount(mu, 0.0)) < 1e-12 * abs(mu[0])
    assert ch.eigencount(mu, 2.0) == pytest.approx(mu[0], rel=1e-14)
    assert mu[0] == pytest.approx(np.sum(p * p) / 8, rel=1e-14)


def test_moments_once_equals_refiltering():
    g = ci.sbm(300, 6, s=10, seed=4)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    p = ch.probe_signals(300, 12, 12, seed=0)
    m = 50
    mu = ch.moments(s, p, m)
    for lam in (0.05, 0.3, 0.77, 1.5):
        assert ch.eigencount(mu, lam) == pytest.approx(ch.eigencount_refilter(s, p, lam, m), rel=1e-11, abs=1e-9)


def test_moments_match_dense_trace_form():
    g = ci.sbm(100, 4, s=6, seed=2)
    lap, w, u = _dense(g)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    p = ch.probe_signals(100, 5, 5, seed=11)
    mu = ch.moments(s, p, 20)
    q = u.T @ p
    for j in range(21):
        ref = np.sum(ch.chebyshev_T(j, w - 1.0)[:, None] * q * q) / 5
        assert mu[j] == pytest.approx(ref, rel=1e-10, abs=1e-10)


def test_dichotomy_rule_on_linear_count():
    lam, c, it, hit = ch.dichotomy(lambda x: 100.0 * x, 37)
    assert hit and ch.round_half_away(c) == 37 and 0.365 <= lam < 0.375
    # an unreachable k collapses the bracket and is flagged
    lam, c, it, hit = ch.dichotomy(lambda x: 0.0 if x < 1.0 else 10.0, 5)
    assert not hit and abs(lam - 1.0) < 1e-11


def test_dichotomy_on_graph_lands_between_eigenvalues():
    g = ci.disjoint_cliques(6, 10)
    s = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    n = g.n
    mu = ch.moments(s, math.sqrt(n) * np.eye(n), 80)
    lam, c, it, hit = ch.dichotomy(lambda x: ch.eigencount(mu, x), 6)
    assert hit and 0.0 < lam < 10 / 9
