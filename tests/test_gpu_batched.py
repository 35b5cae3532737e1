"""Batched CSC: graphs of uneven size (one node, a pair, hubs above the 256-edge
threshold, SBMs, cliques) packed block-diagonally in one handle; every stage is
checked graph by graph against the FP64 oracle run on that graph alone."""
import math

import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import ari as oari
from oracle import chebyshev as och
from oracle import interp as ointerp
from oracle import kmeans as okm
from oracle import laplacian as olap
from oracle import sampling as osamp

from .helpers import rel

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


def _hub(n=1500, seed=0):
    base = ci.sbm(n, 5, s=10.0, seed=seed)
    nbrs = [set(base.col_idx[base.row_ptr[v]:base.row_ptr[v + 1]].tolist()) for v in range(n)]
    for v in range(1, 700):
        nbrs[0].add(v)
        nbrs[v].add(0)
    i = np.concatenate([np.full(len(nb), v) for v, nb in enumerate(nbrs)])
    j = np.concatenate([np.array(sorted(nb), dtype=np.int64) for nb in nbrs])
    return ci.from_edges(n, i, j, labels=base.labels)


BATCH = [
    (ci.sbm(1000, 20, seed=0), 20),
    (ci.from_edges(1, np.array([], np.int64), np.array([], np.int64)), 1),
    (_hub(), 5),
    (ci.ring(33), 3),
    (ci.sbm(600, 6, seed=2), 6),
    (ci.from_edges(2, np.array([0]), np.array([1])), 1),
    (ci.disjoint_cliques(4, 7), 4),
    (ci.erdos_renyi(777, 0.02, seed=3), 8),
]
SIZES = np.array([g.n for g, _ in BATCH])
OFFS = np.concatenate([[0], np.cumsum(SIZES)])
KS = np.array([k for _, k in BATCH], dtype=np.int32)


def _handle():
    return csc.csc_graph_create_batched([(g.row_ptr, g.col_idx) for g, _ in BATCH])


def test_handle_layout():
    with _handle() as h:
        assert h.n_graphs == len(BATCH) and h.N == OFFS[-1]
        assert np.array_equal(csc.csc_graph_degrees(h), np.concatenate([np.diff(g.row_ptr) for g, _ in BATCH]))


def test_moments_per_graph_match_oracle():
    nv, nmom = 12, 41
    probes = och.probe_signals(int(OFFS[-1]), nv, 16, seed=5)  # drawn for the packed rows
    with _handle() as h:
        mu = csc.csc_kpm_moments_batched(h, nmom, nv, seed=5)
    for i, (g, _) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        ref = och.moments(s, probes[OFFS[i]:OFFS[i + 1]], nmom - 1, n_v=nv)
        assert np.max(np.abs(mu[i] - ref)) <= 2e-5 * max(abs(ref[0]), 1e-12), i


def test_lambda_per_graph_is_accepted_by_the_oracle_count():
    nv, m = 12, 50
    probes = och.probe_signals(int(OFFS[-1]), nv, 16, seed=1)
    with _handle() as h:
        lam, infos = csc.csc_estimate_lambda_k_batched(h, KS, m, nv, 1)
    for i, (g, k) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        mu = och.moments(s, probes[OFFS[i]:OFFS[i + 1]], m, n_v=nv)
        if infos[i].hit:
            assert och.round_half_away(och.eigencount(mu, lam[i])) == k, i
        assert infos[i].lam == lam[i]


# Per graph: relative error against the oracle, plus a floor proportional to the
# graph's input (a graph whose filtered block nearly vanishes -- an isolated node
# far from the pass band -- keeps only the storage rounding of its m orders).
FLOOR = {0: 2e-6, 1: 1e-2, 2: 1e-13}


@pytest.mark.parametrize("storage,tol", [(0, 1e-5), (1, 5e-2), (2, 1e-12)])
def test_filter_per_graph_cutoffs_match_oracle(storage, tol):
    d, d_pad, m = 21, 24, 30
    lam = np.linspace(0.2, 1.1, len(BATCH))
    r = ci.gaussian_block(int(OFFS[-1]), d, d_pad, seed=7)
    with _handle() as h:
        y = csc.csc_filter_batched(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                   flags=0).cpu().numpy()
    assert rel(y, np.concatenate([och.cheb_filter(olap.normalized_adjacency(g.row_ptr, g.col_idx),
                                                  r[OFFS[i]:OFFS[i + 1]].astype(np.float64),
                                                  och.filter_coeffs(lam[i], m))
                                  for i, (g, _) in enumerate(BATCH)])) <= tol
    for i, (g, _) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        ri = r[OFFS[i]:OFFS[i + 1]].astype(np.float64)
        ref = och.cheb_filter(s, ri, och.filter_coeffs(lam[i], m))
        err = np.linalg.norm(y[OFFS[i]:OFFS[i + 1]] - ref)
        assert err <= tol * np.linalg.norm(ref) + FLOOR[storage] * np.linalg.norm(ri), i


@pytest.mark.parametrize("G,NT,tiles", [(2, 1, 3), (4, 3, 1), (32, 1, 1)])
def test_filter_pinned_shapes_batched(G, NT, tiles):
    d, d_pad, m = 21, 24, 12
    lam = np.linspace(0.3, 0.9, len(BATCH))
    r = ci.gaussian_block(int(OFFS[-1]), d, d_pad, seed=8)
    with _handle() as h:
        with pytest.raises(csc.CscError):  # fewer ranges than graphs
            csc.csc_graph_pin_shape(h, "cheb_step", 4, d_pad, G, NT, 256, len(BATCH) - 1, tiles, 0)
            csc.csc_filter_batched(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=0)
    with _handle() as h:
        csc.csc_graph_pin_shape(h, "cheb_step", 4, d_pad, G, NT, 256, 29, tiles, 0)
        y = csc.csc_filter_batched(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=0).cpu().numpy()
    for i, (g, _) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        ref = och.cheb_filter(s, r[OFFS[i]:OFFS[i + 1]].astype(np.float64), och.filter_coeffs(lam[i], m))
        assert rel(y[OFFS[i]:OFFS[i + 1]], ref) <= 1e-5, i


def test_sample_per_graph_bit_exact():
    n = np.array([min(g.n, max(1, math.ceil(2 * k * math.log(k))) if k > 1 else 1) for g, k in BATCH])
    n[3] = 0  # a graph may contribute no sample
    with _handle() as h:
        idx = csc.csc_sample_batched(h, n, seed=11).cpu().numpy()
    ref = np.concatenate([osamp.sample(int(SIZES[i]), int(n[i]), 11 + i) + OFFS[i] for i in range(len(BATCH))])
    assert np.array_equal(idx, ref)


def test_kmeans_per_problem_matches_oracle():
    rng = np.random.default_rng(3)
    ns, ks = [120, 1, 40, 7, 300], [20, 1, 5, 7, 9]
    xs = [rng.standard_normal((n, 28)).astype(np.float32) for n in ns]
    x = np.zeros((sum(ns), 32), np.float32)
    x[:, :28] = np.concatenate(xs)
    lab, inertia = csc.csc_kmeans_batched(torch.from_numpy(x).cuda(), ns, ks, d=28, replicates=5, seed=4)
    lab = lab.cpu().numpy()
    off = 0
    for i, (n, k) in enumerate(zip(ns, ks)):
        lr, _, ir, _ = okm.kmeans(xs[i].astype(np.float64), k, 5, 100, seed=4 + i)
        assert inertia[i] == pytest.approx(ir, rel=1e-4, abs=1e-9)
        assert oari.ari(lab[off:off + n], lr) >= 0.99 or n == k
        off += n


def test_interpolation_per_graph_matches_oracle():
    gamma, power = 1e-3, 4
    n = [min(g.n, max(k, math.ceil(2 * k * math.log(k))) if k > 1 else 1) for g, k in BATCH]
    oms = [osamp.sample(g.n, n[i], 2 + i) for i, (g, _) in enumerate(BATCH)]
    labs = [(g.labels[om] if g.labels is not None else om % k).astype(np.int32) for (g, k), om in zip(BATCH, oms)]
    idx = np.concatenate([om + OFFS[i] for i, om in enumerate(oms)])
    with _handle() as h:
        labels, fz, info = csc.csc_interpolate_batched(h, torch.from_numpy(idx).cuda(),
                                                       torch.from_numpy(np.concatenate(labs)).cuda(), KS, power,
                                                       gamma, 1e-7, 5000, fuzzy=True)
    assert info.converged
    labels, fz = labels.cpu().numpy(), fz.cpu().numpy()
    for i, (g, k) in enumerate(BATCH):
        lap = olap.laplacian(g.row_ptr, g.col_idx)
        x_ref, _, _ = ointerp.interpolate(lap, oms[i], labs[i], k, gamma, power, tol=1e-11)
        x = fz[OFFS[i]:OFFS[i + 1], :k].astype(np.float64)
        # the residual, recomputed by the oracle in fp64, and the forward error it bounds
        b = ointerp.rhs(g.n, oms[i], labs[i], k)
        msk = ointerp.mask(g.n, oms[i])
        res = ointerp.apply_system(lap, msk, gamma, power, x) - b
        rres = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
        assert np.max(rres) <= 3e-6, i
        kappa = np.linalg.cond(ointerp.system_matrix(lap, msk, gamma, power).toarray())
        err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
        assert np.all(err <= kappa * rres * (1 + 1e-6) + 1e-9), i
        if kappa < 1e4:
            assert rel(x, x_ref) <= 1e-3, i
        assert np.array_equal(labels[OFFS[i]:OFFS[i + 1]], ointerp.labels_from_indicators(x)), i


def test_cluster_batched_matches_separate_runs():
    """Per-graph ARI against the planted communities of the batched pipeline equals
    that of one csc_cluster call per graph."""
    graphs = [(ci.sbm(n, k, seed=10 + i), k) for i, (n, k) in
              enumerate([(2000, 10), (3000, 30), (1200, 6), (5000, 50), (800, 8), (2500, 25)])]
    with csc.csc_graph_create_batched([(g.row_ptr, g.col_idx) for g, _ in graphs]) as h:
        labels, lam, info = csc.csc_cluster_batched(h, [k for _, k in graphs], seed=0)
    labels = labels.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([g.n for g, _ in graphs])])
    assert info.lambda_hits == len(graphs) and info.cg.converged
    a_b, a_s = [], []
    for i, (g, k) in enumerate(graphs):
        lb = labels[offs[i]:offs[i + 1]]
        assert lb.min() >= 0 and lb.max() < k
        a_b.append(oari.ari(lb, g.labels))
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h1:
            l1, _ = csc.csc_cluster(h1, k, seed=i)
        a_s.append(oari.ari(l1.cpu().numpy(), g.labels))
    assert abs(np.mean(a_b) - np.mean(a_s)) <= 0.03
    assert np.mean(a_b) >= 0.8


@pytest.mark.parametrize("storage,tol", [(0, 1e-5), (2, 1e-12)])
def test_clenshaw_per_graph_cutoffs_match_oracle(storage, tol):
    d, d_pad, m = 21, 24, 30
    lam = np.linspace(0.2, 1.1, len(BATCH))
    r = ci.gaussian_block(int(OFFS[-1]), d, d_pad, seed=7)
    with _handle() as h:
        y = csc.csc_filter_batched(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                   flags=csc.CLENSHAW).cpu().numpy()
    for i, (g, _) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        ri = r[OFFS[i]:OFFS[i + 1]].astype(np.float64)
        ref = och.cheb_filter(s, ri, och.filter_coeffs(lam[i], m))
        err = np.linalg.norm(y[OFFS[i]:OFFS[i + 1]] - ref)
        assert err <= tol * np.linalg.norm(ref) + FLOOR[storage] * np.linalg.norm(ri), i


def test_interpolation_highpass_per_graph_matches_oracle():
    """Each graph's systems use g = 1 - h~ at its own cut-off; the residual recomputed
    by the oracle's high-pass operator on that graph alone."""
    gamma, m = 1e-3, 30
    lam = np.linspace(0.25, 0.9, len(BATCH))
    n = [min(g.n, max(k, math.ceil(2 * k * math.log(k))) if k > 1 else 1) for g, k in BATCH]
    oms = [osamp.sample(g.n, n[i], 5 + i) for i, (g, _) in enumerate(BATCH)]
    labs = [(g.labels[om] if g.labels is not None else om % k).astype(np.int32) for (g, k), om in zip(BATCH, oms)]
    idx = np.concatenate([om + OFFS[i] for i, om in enumerate(oms)])
    with _handle() as h:
        labels, fz, info = csc.csc_interpolate_batched_highpass(h, torch.from_numpy(idx).cuda(),
                                                                torch.from_numpy(np.concatenate(labs)).cuda(), KS,
                                                                lam, m, gamma, 1e-7, 5000, fuzzy=True)
    assert info.converged
    labels, fz = labels.cpu().numpy(), fz.cpu().numpy()
    for i, (g, k) in enumerate(BATCH):
        s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
        x = fz[OFFS[i]:OFFS[i + 1], :k].astype(np.float64)
        b = ointerp.rhs(g.n, oms[i], labs[i], k)
        res = ointerp.apply_highpass(s, ointerp.mask(g.n, oms[i]), gamma, lam[i], m, x) - b
        bn = np.linalg.norm(b, axis=0)
        # a cluster with no sample has b = 0 and the solution 0: its residual is checked absolutely
        rres = np.linalg.norm(res, axis=0) / np.where(bn > 0, bn, 1.0)
        assert np.max(rres) <= 3e-6, i
        assert np.all(x[:, bn == 0] == 0), i
        assert np.array_equal(labels[OFFS[i]:OFFS[i + 1]], ointerp.labels_from_indicators(x)), i


def test_cluster_batched_highpass_matches_separate_runs():
    gs = [ci.sbm(n, k, seed=10 + i) for i, (n, k) in enumerate([(1200, 12), (2000, 20), (900, 9), (3000, 15)])]
    ks = [12, 20, 9, 15]
    with csc.csc_graph_create_batched([(g.row_ptr, g.col_idx) for g in gs]) as h:
        lb, lam, info = csc.csc_cluster_batched(h, ks, seed=3, flags=csc.HIGHPASS)
    assert info.cg.converged
    lb = lb.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    a_b, a_s = [], []
    for i, (g, k) in enumerate(zip(gs, ks)):
        a_b.append(oari.ari(lb[offs[i]:offs[i + 1]], g.labels))
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h1:
            l1, i1 = csc.csc_cluster(h1, k, seed=3 + i, flags=csc.HIGHPASS)
        a_s.append(oari.ari(l1.cpu().numpy(), g.labels))
    assert abs(np.mean(a_b) - np.mean(a_s)) <= 0.03
    assert np.mean(a_b) >= 0.85
