"""Pins of the oracle's spectral clustering (Alg. 1), the baseline of the recovery sweeps."""
import numpy as np
import scipy.sparse.linalg as sla

import csc_inputs as ci
from oracle import ari, laplacian, sc


def test_cliques_recovered_exactly():
    g = ci.disjoint_cliques(5, 9)
    lab, ev = sc.spectral_clustering(g.row_ptr, g.col_idx, 5, seed=1)
    assert ari.ari(lab, g.labels) == 1.0
    assert np.allclose(ev[:5], 0.0, atol=1e-12) and ev[5] > 0.5


def test_sbm_without_cross_edges_recovered_exactly():
    g = ci.sbm(600, 6, s=12.0, eps=0.0, seed=3)
    lab, ev = sc.spectral_clustering(g.row_ptr, g.col_idx, 6, seed=0)
    assert ari.ari(lab, g.labels) == 1.0


def test_eigenspace_matches_arpack():
    g = ci.sbm(400, 4, s=10.0, seed=2)
    ev, u = sc.spectrum(g.row_ptr, g.col_idx)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    w, v = sla.eigsh(lap, k=4, sigma=-1e-3, which="LM")
    assert np.allclose(np.sort(w), ev[:4], atol=1e-9)
    # principal angles between the two 4-dimensional subspaces are all ~0
    s = np.linalg.svd(u[:, :4].T @ np.linalg.qr(v)[0], compute_uv=False)
    assert np.all(s > 1 - 1e-8)


def test_two_communities_match_fiedler_signs():
    g = ci.sbm(300, 2, s=12.0, seed=4)
    lab, _ = sc.spectral_clustering(g.row_ptr, g.col_idx, 2, seed=0)
    _, u = sc.spectrum(g.row_ptr, g.col_idx)
    fiedler = (u[:, 1] > 0).astype(int)
    assert ari.ari(lab, fiedler) > 0.95


def test_features_unit_rows_and_zero_row():
    u = np.array([[3.0, 4.0], [0.0, 0.0], [1.0, 0.0]])
    f = sc.features(u)
    assert np.allclose(f, [[0.6, 0.8], [0.0, 0.0], [1.0, 0.0]])
