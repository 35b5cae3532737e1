"""Pins of the oracle's sampling (Eq. 4), k-means (Alg. 2 step 6), interpolation (Eq. 5),
label rule (Sec. 4.1) and ARI (Sec. 5.2)."""
import itertools

import numpy as np
import pytest
from scipy import stats

import csc_inputs as ci
from oracle import ari, interp, kmeans, laplacian, sampling


# --- sampling -------------------------------------------------------------

@pytest.mark.parametrize("n_nodes,n", [(1, 1), (10, 0), (10, 10), (1000, 120), (5, 3)])
def test_sample_shape(n_nodes, n):
    om = sampling.sample(n_nodes, n, seed=3)
    assert om.dtype == np.int64 and len(om) == n
    assert np.all(np.diff(om) > 0)
    assert np.all((om >= 0) & (om < n_nodes))
    m = sampling.sampling_matrix(n_nodes, om)
    assert np.all(m.sum(axis=1) == 1)


def test_sample_uniform_inclusion():
    n_nodes, n, trials = 50, 10, 4000
    hits = np.zeros(n_nodes)
    for s in range(trials):
        hits[sampling.sample(n_nodes, n, seed=s)] += 1
    expected = trials * n / n_nodes
    chi2 = np.sum((hits - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, n_nodes - 1) > 1e-3


def test_sample_invalid():
    with pytest.raises(ValueError):
        sampling.sample(5, 6, 0)


# --- k-means --------------------------------------------------------------

def _brute_force_inertia(x, k):
    best = np.inf
    n = len(x)
    for assign in itertools.product(range(k), repeat=n):
        a = np.array(assign)
        if len(set(assign)) < k:
            continue
        tot = 0.0
        for j in range(k):
            pts = x[a == j]
            tot += np.sum((pts - pts.mean(axis=0)) ** 2)
        best = min(best, tot)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_kmeans_reaches_brute_force_optimum(seed):
    rng = np.random.default_rng(seed)
    k = 2 + seed % 2
    x = rng.normal(size=(8, 2)) + np.repeat(rng.normal(scale=3, size=(k, 2)), [3, 3, 2][:k] if k == 3 else [4, 4], axis=0)
    lab, c, inertia, _ = kmeans.kmeans(x, k, replicates=20, max_iter=100, seed=seed)
    assert inertia == pytest.approx(_brute_force_inertia(x, k), rel=1e-12)


def test_kmeans_fixed_point_and_blobs():
    rng = np.random.default_rng(0)
    centers = rng.normal(scale=10, size=(5, 3))
    truth = np.repeat(np.arange(5), 20)
    x = centers[truth] + rng.normal(scale=0.1, size=(100, 3))
    lab, c, inertia, _ = kmeans.kmeans(x, 5, replicates=20, max_iter=100, seed=1)
    assert ari.ari(lab, truth) == 1.0
    d = np.sum((x[:, None] - c[None]) ** 2, axis=2)
    assert np.array_equal(np.argmin(d, axis=1), lab)
    for j in range(5):
        assert np.allclose(c[j], x[lab == j].mean(axis=0))


# --- interpolation ----------------------------------------------------------

def test_interp_matches_dense_solve():
    g = ci.sbm(200, 4, s=8, seed=1)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    om = sampling.sample(200, 30, seed=2)
    lab = g.labels[om]
    x, it, res = interp.interpolate(lap, om, lab, 4, gamma=1e-3, power=4, tol=1e-12)
    ref = interp.interpolate_dense(lap.toarray(), om, lab, 4, 1e-3, 4)
    assert res < 1e-11
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8


def test_interp_full_sampling_small_gamma_returns_observations():
    g = ci.sbm(60, 3, s=6, seed=0)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    om = np.arange(60)
    lab = g.labels
    x, _, _ = interp.interpolate(lap, om, lab, 3, gamma=1e-9, power=4, tol=1e-13)
    assert np.allclose(x, interp.rhs(60, om, lab, 3), atol=1e-7)


def test_interp_disjoint_regular_cliques_exact():
    g = ci.disjoint_cliques(4, 7)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    om = np.array([0, 9, 15, 27])
    lab = g.labels[om]
    x, _, res = interp.interpolate(lap, om, lab, 4, gamma=1e-3, power=4, tol=1e-13)
    truth = np.eye(4)[g.labels]
    assert np.allclose(x, truth, atol=1e-9)
    assert np.array_equal(interp.labels_from_indicators(x), g.labels)


def test_interp_highpass_matches_eigendecomposition():
    """g = 1 - h~ applied by the Chebyshev recurrence equals U (1 - h~(Lambda)) U^T."""
    g = ci.sbm(200, 4, s=8, seed=1)
    s_mat = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    om = sampling.sample(200, 30, seed=2)
    lab = g.labels[om]
    x, it, res = interp.interpolate_highpass(s_mat, om, lab, 4, lam=0.3, m=30, gamma=1e-2, tol=1e-12)
    ref = interp.interpolate_highpass_dense(lap.toarray(), om, lab, 4, 0.3, 30, 1e-2)
    assert res < 1e-11
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8


def test_interp_highpass_cliques_near_exact():
    """Indicators of disjoint cliques span the eigenvalue 0 where h~ = 1 up to the
    Jackson error, so every clique sampled recovers them within gamma times that error."""
    g = ci.disjoint_cliques(4, 7)
    s_mat = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    om = np.array([0, 9, 15, 27])
    lab = g.labels[om]
    x, _, _ = interp.interpolate_highpass(s_mat, om, lab, 4, lam=0.5, m=50, gamma=1e-3, tol=1e-13)
    truth = np.eye(4)[g.labels]
    assert np.max(np.abs(x - truth)) < 1e-3
    assert np.array_equal(interp.labels_from_indicators(x), g.labels)


def test_label_rule_normalises_and_breaks_ties_low():
    x = np.array([[1.0, 2.0], [1.0, 0.0], [0.0, 0.0]])
    # column norms sqrt(2) and 2: row 0 -> 0.707 vs 1.0 -> 1; row 2 tie -> 0
    assert list(interp.labels_from_indicators(x)) == [1, 0, 0]


# --- ARI ----------------------------------------------------------------------

def test_ari_pins():
    a = [0, 0, 0, 1, 1, 1]
    b = [0, 0, 1, 1, 2, 2]
    assert ari.ari(a, b) == pytest.approx(8 / 33, rel=1e-14)
    assert ari.ari(a, a) == 1.0
    assert ari.ari([0, 0, 1, 1], [5, 5, 2, 2]) == 1.0
    assert ari.ari([0, 0, 0, 0], [0, 1, 2, 3]) == 0.0
    rng = np.random.default_rng(0)
    u = rng.integers(0, 5, 300)
    v = rng.integers(0, 5, 300)
    perm = np.array([3, 1, 4, 0, 2])
    assert ari.ari(u, v) == pytest.approx(ari.ari(perm[u], v), abs=1e-15)
    assert abs(ari.ari(u, v)) < 0.05


@pytest.mark.parametrize("k,size,n", [(6, 12, 36), (4, 25, 30), (10, 8, 60)])
def test_pipeline_exact_on_disjoint_cliques(k, size, n):
    """Alg. 2 end to end where the answer is fixed: k disjoint cliques have lambda_1..k = 0
    and lambda_k+1 = size/(size-1), so the eigencount stops inside the gap, the filtered
    features are the clique indicators, and every clique holding a sample is recovered."""
    from oracle import pipeline

    g = ci.disjoint_cliques(k, size)
    out = pipeline.csc(g.row_ptr, g.col_idx, k, seed=3, n=n, replicates=5)
    assert out["est"]["hit"] and 0.0 < out["lam"] < size / (size - 1)
    assert len(set(g.labels[out["omega"]])) == k
    assert ari.ari(out["labels"], g.labels) == 1.0
