"""Alg. 2 end to end through csc_cluster against the oracle pipeline (ARI within 0.01),
and the full-size SBM workload (N = 1e5, k = 200) against the oracle's stored run and
through properties the oracle checks."""
import hashlib
import os

import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import ari as oari
from oracle import chebyshev as och
from oracle import interp as ointerp
from oracle import laplacian as olap
from oracle import pipeline as opipe
from oracle import sampling as osamp

from .helpers import rel

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("rcm", [0, 1, 8, 9])  # graph flags: none, RCM, degree order, both
def test_csc_sbm_1e3_matches_oracle(seed, rcm):
    g = ci.sbm(1000, 20, seed=seed)
    ref = opipe.csc(g.row_ptr, g.col_idx, 20, seed=seed)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, rcm) as h:
        labels, info = csc.csc_cluster(h, 20, seed=seed)
    lab = labels.cpu().numpy()
    a_gpu = oari.ari(lab, g.labels)
    a_ref = oari.ari(ref["labels"], g.labels)
    assert abs(a_gpu - a_ref) <= 0.01
    assert oari.ari(lab, ref["labels"]) >= 0.98
    assert info.lam.hit and abs(info.lam.lam - ref["lam"]) < 1e-9 + 2.0 ** -info.lam.iters
    assert info.inertia == pytest.approx(ref["inertia"], rel=1e-3)


@pytest.mark.parametrize("storage", [1, 2])  # BF16, F64
def test_csc_sbm_1e3_storage_variants(storage):
    g = ci.sbm(1000, 20, seed=0)
    ref = opipe.csc(g.row_ptr, g.col_idx, 20, seed=0)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, 20, seed=0, storage=storage)
    a_gpu = oari.ari(labels.cpu().numpy(), g.labels)
    a_ref = oari.ari(ref["labels"], g.labels)
    assert abs(a_gpu - a_ref) <= 0.01


def test_csc_edge_cases():
    # k = 1: every node in cluster 0
    g = ci.sbm(200, 4, s=10, seed=1)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, 1, seed=0)
        assert torch.all(labels == 0)
    # disjoint cliques are recovered exactly
    g = ci.disjoint_cliques(6, 12)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, 6, seed=3, n=36)
    assert oari.ari(labels.cpu().numpy(), g.labels) == 1.0


def test_csc_full_size_sbm_1e5():
    """N = 1e5, k = 200, d = 47 -> 48, m = 50, n = 2120: every stage checked by the oracle
    where it finishes in seconds (features, sampling, the CG residual, the label rule)."""
    g = ci.sbm(100_000, 200, seed=0)
    k, seed = 200, 0
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, k, seed=seed)
        lam = info.lam.lam
        feats = csc.csc_filter_random_signals(h, lam, 50, 47, 48, seed=seed).cpu().numpy()
        om = csc.csc_sample(g.n, 2120, seed).cpu().numpy()
        lab_r, _ = csc.csc_kmeans_reduced(torch.from_numpy(np.ascontiguousarray(feats[om])).cuda(), 47, k, 20, 100,
                                          seed)
        lab2, fz, cg = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), lab_r, k, fuzzy=True)
    lab = labels.cpu().numpy()
    # lambda_k: a valid dichotomy answer under the oracle's moments
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    mu = och.moments(s, och.probe_signals(g.n, 24, 24, seed), 50)
    assert abs(och.eigencount(mu, lam) - k) < 0.5 + 1e-2
    # features vs the oracle filter of the same Philox block
    ref = och.normalize_rows(och.cheb_filter(s, och.random_signals(g.n, 47, 48, seed), och.filter_coeffs(lam, 50)))
    assert rel(feats, ref) <= 1e-5
    assert np.array_equal(om, osamp.sample(g.n, 2120, seed))
    # CG residual recomputed in fp64 by the oracle
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    lr = lab_r.cpu().numpy()
    b = ointerp.rhs(g.n, om, lr, k)
    x = fz.cpu().numpy().astype(np.float64)
    res = ointerp.apply_system(lap, ointerp.mask(g.n, om), 1e-3, 4, x) - b
    assert cg.converged
    assert np.max(np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)) <= 3e-6
    assert np.array_equal(lab2.cpu().numpy(), ointerp.labels_from_indicators(fz.cpu().numpy()))
    assert np.array_equal(lab, lab2.cpu().numpy())
    # recovery of the planted partition (the oracle pipeline scores ~0.86 on this graph)
    assert oari.ari(lab, g.labels) >= 0.8


GOLDEN_C2 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "csc_sbm_n1e5_k200_seed0.npz")


def test_csc_sbm_1e5_k200_against_oracle_run():
    """The SBM with N = 1e5, k = 200 (mean degree 16, eps = eps_c / 4, seed 0; d = 47, m = 50,
    n = 2120, L^4 with gamma = 1e-3) end to end against the FP64 oracle's run of Alg. 2,
    written by tests/golden/make_csc_sbm_n1e5_k200.py: the ARI against the planted
    communities within 0.01 of the oracle's, the labels' own agreement with the oracle's
    (ARI) reported and bounded, and the same lambda_k (same probes, same dichotomy)."""
    ref = np.load(GOLDEN_C2)
    g = ci.sbm(100_000, 200, seed=0)
    hh = hashlib.sha256()
    hh.update(np.ascontiguousarray(g.row_ptr, dtype=np.int64).tobytes())
    hh.update(np.ascontiguousarray(g.col_idx, dtype=np.int32).tobytes())
    assert g.nnz == int(ref["nnz"]) and hh.hexdigest() == str(ref["csr_sha256"]), "graph generator changed"
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, 200, seed=0)
    lab = labels.cpu().numpy()
    a_gpu = oari.ari(lab, g.labels)
    a_ref = float(ref["ari_vs_planted"])
    agree = oari.ari(lab, ref["labels"].astype(np.int64))
    print(f"ARI vs planted: GPU {a_gpu:.4f}, oracle {a_ref:.4f}; ARI(GPU labels, oracle labels) {agree:.4f}")
    assert abs(a_gpu - a_ref) <= 0.01, f"ARI {a_gpu:.4f} vs oracle {a_ref:.4f}"
    assert agree >= 0.9, f"ARI between the GPU and oracle labels {agree:.4f}"
    assert info.lam.hit and abs(info.lam.lam - float(ref["lam"])) < 1e-9 + 2.0 ** -info.lam.iters


def test_eigencount_degree_parameter():
    """m_count sets the degree of step 1's eigencount filter only: csc_cluster's lambda_k is
    csc_estimate_lambda_k's at that degree, a valid dichotomy answer for the oracle's moments."""
    g = ci.sbm(1000, 20, seed=1)
    ref = opipe.csc(g.row_ptr, g.col_idx, 20, seed=1, m_count=150)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        est = csc.csc_estimate_lambda_k(h, 20, 150, seed=1)
        labels, info = csc.csc_cluster(h, 20, seed=1, m_count=150)
        _, info50 = csc.csc_cluster(h, 20, seed=1)
    assert info.lam.lam == est.lam and info.lam.m == 150 and info50.lam.m == 50
    assert info.lam.hit and abs(info.lam.lam - ref["lam"]) < 1e-9 + 2.0 ** -info.lam.iters
    assert oari.ari(labels.cpu().numpy(), g.labels) >= 0.9


def test_eigencount_degree_parameter_batched():
    gs = [ci.sbm(600, 6, seed=i) for i in range(3)]
    with csc.csc_graph_create_batched([(g.row_ptr, g.col_idx) for g in gs]) as h:
        lam_ref, _ = csc.csc_estimate_lambda_k_batched(h, [6, 6, 6], 120)
        _, lam, info = csc.csc_cluster_batched(h, [6, 6, 6], m_count=120)
    assert np.array_equal(lam, lam_ref)
