"""Parity of the eigencount moments and lambda_k estimate (Sec. 4.3), sampling (Eq. 4),
reduced k-means (Alg. 2 step 6) and interpolation (Eq. 5, Sec. 4.1) with the oracle."""
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
from paper_1602_02018_gb300 import _native as nat  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


# ------------------------------------------------------------------ moments

@pytest.mark.parametrize("n,k,n_mom,n_v,rcm", [(1000, 20, 51, 14, False), (1000, 20, 51, 14, True),
                                               (1000, 20, 51, 14, 9),
                                               (777, 7, 64, 8, False), (2000, 10, 2, 3, False),
                                               (300, 6, 1, 5, False), (300, 6, 12, 17, True)])
def test_moments_match_oracle(n, k, n_mom, n_v, rcm):
    g = ci.sbm(n, k, s=12.0, seed=3) if n % k == 0 else ci.erdos_renyi(n, 12.0 / n, seed=3)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    probes = och.probe_signals(g.n, n_v, n_v, seed=17)
    ref = och.moments(s, probes, max(n_mom - 1, 0))[:n_mom]
    with csc.csc_graph_create(g.row_ptr, g.col_idx, int(rcm)) as h:
        mu = csc.csc_kpm_moments(h, n_mom, n_v, seed=17)
    assert np.max(np.abs(mu - ref)) <= 2e-5 * abs(ref[0])


def test_moments_bf16_bound():
    g = ci.sbm(1000, 20, seed=0)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    ref = och.moments(s, och.probe_signals(g.n, 14, 14, seed=1), 50)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        mu = csc.csc_kpm_moments(h, 51, 14, seed=1, storage=csc.BF16)
    assert np.max(np.abs(mu - ref)) <= 2e-2 * ref[0]


@pytest.mark.parametrize("n,k,seed", [(1000, 20, 0), (1000, 20, 5), (3000, 30, 1)])
def test_lambda_k_matches_oracle(n, k, seed):
    g = ci.sbm(n, k, seed=seed)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    n_v = math.ceil(2 * math.log(n))
    est = och.estimate_lambda_k(s, k, 50, n_v, seed)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        info = csc.csc_estimate_lambda_k(h, k, 50, 0, seed)
    assert info.n_probes == n_v and info.moment_passes == 25
    assert info.hit == est["hit"]
    # the GPU's lambda is a valid dichotomy answer under the oracle's moments
    c = och.eigencount(est["mu"], info.lam)
    assert abs(c - k) < 0.5 + 1e-3
    assert abs(info.lam - est["lam"]) <= 2.0 ** -info.iters + 1e-12 or info.lam == est["lam"]


def test_lambda_k_bracket():
    g = ci.sbm(1000, 20, seed=0)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        base = csc.csc_estimate_lambda_k(h, 20, 50, 0, 0)
        good = csc.csc_estimate_lambda_k(h, 20, 50, 0, 0, bracket=(base.lam - 0.05, base.lam + 0.05))
        bad = csc.csc_estimate_lambda_k(h, 20, 50, 0, 0, bracket=(1.5, 1.9))
    assert good.bracket_used and round(good.count) == 20
    assert not bad.bracket_used and bad.lam == base.lam


# ----------------------------------------------------------------- sampling

@pytest.mark.parametrize("N,n,seed", [(1, 1, 0), (10, 10, 1), (1000, 120, 0), (100_000, 2_120, 0),
                                      (12_345, 1, 7), (65_537, 922, 2**63 + 5), (5_000, 4_999, 3),
                                      (1_000_000, 922, 0)])
def test_sample_bit_exact(N, n, seed):
    got = csc.csc_sample(N, n, seed).cpu().numpy()
    assert np.array_equal(got, osamp.sample(N, n, seed))


def test_sample_zero():
    out = csc.csc_sample(100, 0, 1)
    assert out.numel() == 0


# ------------------------------------------------------------------ k-means

def _features(n_nodes=1000, k=20, seed=0):
    g = ci.sbm(n_nodes, k, seed=seed)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    r = och.random_signals(g.n, 28, 28, seed)
    f = och.normalize_rows(och.cheb_filter(s, r, och.filter_coeffs(0.44, 50)))
    om = osamp.sample(g.n, 120, seed)
    return f[om].astype(np.float32)


@pytest.mark.parametrize("k,reps", [(20, 20), (20, 1), (5, 3)])
def test_kmeans_matches_oracle(k, reps):
    x = _features()
    lab_ref, _, in_ref, _ = okm.kmeans(x.astype(np.float64), k, reps, 100, seed=4)
    xt = torch.zeros((x.shape[0], 32), dtype=torch.float32, device="cuda")
    xt[:, :28] = torch.from_numpy(x).cuda()
    lab, inertia = csc.csc_kmeans_reduced(xt, 28, k, reps, 100, seed=4)
    lab = lab.cpu().numpy()
    assert inertia == pytest.approx(in_ref, rel=1e-4)
    assert oari.ari(lab, lab_ref) >= 0.99


def test_kmeans_separated_blobs_and_edge_cases():
    rng = np.random.default_rng(0)
    centers = rng.normal(scale=10, size=(7, 5))
    truth = np.repeat(np.arange(7), 30)
    x = (centers[truth] + rng.normal(scale=0.05, size=(210, 5))).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    lab, inertia = csc.csc_kmeans_reduced(xt, 5, 7, 20, 100, seed=1)
    assert oari.ari(lab.cpu().numpy(), truth) == 1.0
    # k = 1 and n == k
    lab1, in1 = csc.csc_kmeans_reduced(xt, 5, 1, 2, 10, seed=0)
    assert torch.all(lab1 == 0)
    assert in1 == pytest.approx(float(np.sum((x - x.mean(axis=0)) ** 2)), rel=1e-5)
    labn, inn = csc.csc_kmeans_reduced(xt[:7].contiguous(), 5, 7, 3, 10, seed=0)
    assert sorted(labn.cpu().tolist()) == list(range(7)) and inn == 0.0


# ------------------------------------------------------------ interpolation

@pytest.mark.parametrize("n_nodes,k,n_s,power,rcm", [(1000, 20, 120, 4, False), (1000, 20, 120, 4, True),
                                                     (1000, 20, 120, 4, 9),
                                                   (600, 6, 40, 2, False), (500, 5, 30, 1, False)])
def test_interpolation_matches_oracle(n_nodes, k, n_s, power, rcm):
    g = ci.sbm(n_nodes, k, seed=2)
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    om = osamp.sample(g.n, n_s, 2)
    lab = g.labels[om].astype(np.int32)
    x_ref, _, _ = ointerp.interpolate(lap, om, lab, k, 1e-3, power, tol=1e-11)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, int(rcm)) as h:
        labels, fz, info = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), k,
                                               power, 1e-3, 1e-7, 5000, fuzzy=True)
    assert info.converged and info.max_rel_residual <= 1e-6
    x = fz.cpu().numpy()
    # the residual, recomputed by the oracle in fp64
    b = ointerp.rhs(g.n, om, lab, k)
    msk = ointerp.mask(g.n, om)
    res = ointerp.apply_system(lap, msk, 1e-3, power, x.astype(np.float64)) - b
    rres = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    assert np.max(rres) <= 3e-6
    # forward error bound: ||x - x*|| / ||x*|| <= cond(A) ||b - A x|| / ||b|| per column
    a = ointerp.system_matrix(lap, msk, 1e-3, power).toarray()
    kappa = np.linalg.cond(a)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert np.all(err <= kappa * rres * (1 + 1e-6) + 1e-9)
    assert rel(x, x_ref) <= 1e-3
    assert np.array_equal(labels.cpu().numpy(), ointerp.labels_from_indicators(x))
    assert oari.ari(labels.cpu().numpy(), ointerp.labels_from_indicators(x_ref)) >= 0.999


def test_interpolation_cliques_exact():
    g = ci.disjoint_cliques(4, 7)
    om = np.array([0, 9, 15, 27], dtype=np.int64)
    lab = g.labels[om].astype(np.int32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, fz, info = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), 4,
                                               fuzzy=True)
    assert np.array_equal(labels.cpu().numpy(), g.labels)
    assert np.allclose(fz.cpu().numpy(), np.eye(4)[g.labels], atol=1e-5)


def test_interpolation_not_converged_status():
    g = ci.sbm(1000, 20, seed=2)
    om = osamp.sample(g.n, 120, 2)
    lab = g.labels[om].astype(np.int32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, _, info = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), 20,
                                              max_iter=3)
    assert not info.converged and info.iters == 3


def test_interpolation_bad_label_rejected():
    g = ci.sbm(100, 5, s=8, seed=2)
    om = np.array([0, 50], dtype=np.int64)
    lab = np.array([0, 7], dtype=np.int32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        with pytest.raises(csc.CscError):
            csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), 5)


@pytest.mark.parametrize("G,NT,lean", [(2, 1, 0), (4, 1, 0), (8, 1, 0), (16, 1, 0), (16, 2, 0), (32, 1, 0), (32, 2, 0),
                                       (2, 1, 1), (4, 1, 1), (8, 1, 1), (16, 1, 1), (32, 1, 1)])
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("global_index", [0, 1])
def test_interpolation_every_cg_shape(G, NT, lean, threads, global_index):
    g = ci.sbm(600, 6, seed=2)
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    om = osamp.sample(g.n, 40, 2)
    lab = g.labels[om].astype(np.int32)
    k, ld = 6, 8
    tiles = -(-(ld // 4) // (G * NT))
    x_ref, _, _ = ointerp.interpolate(lap, om, lab, k, 1e-3, 4, tol=1e-11)
    if lean and threads != 256:
        pytest.skip("the lean form runs 256 threads")
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_graph_pin_shape(h, "cg", 4, ld, G, NT, threads, 23, tiles, global_index, lean)
        labels, fz, info = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), k,
                                               4, 1e-3, 1e-7, 5000, fuzzy=True)
    assert info.converged
    assert rel(fz.cpu().numpy(), x_ref) <= 1e-3


def test_interpolation_graph_replay_matches_eager():
    """CG iterations replayed from captured CUDA graphs give the eager launches' bits."""
    g = ci.sbm(1000, 20, seed=2)
    om = osamp.sample(g.n, 120, 2)
    lab = torch.from_numpy(g.labels[om].astype(np.int32)).cuda()
    omd = torch.from_numpy(om).cuda()
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_profile_enable(True)
        l0, f0, i0 = csc.csc_interpolate(h, omd, lab, 20, fuzzy=True)
        csc.csc_profile_enable(False)
        l1, f1, i1 = csc.csc_interpolate(h, omd, lab, 20, fuzzy=True)
        l2, f2, i2 = csc.csc_interpolate(h, omd, lab, 20, fuzzy=True)
    assert i0.iters == i1.iters == i2.iters
    assert torch.equal(f0, f1) and torch.equal(f1, f2) and torch.equal(l0, l2)


def test_interpolation_column_compaction():
    """Columns whose CG has converged leave the iteration (the active ones are moved to the
    front slots): on a power-law graph the columns converge hundreds of iterations apart,
    so the solve compacts; every column must still meet the residual target (recomputed by
    the oracle), keep its place, and the replayed graphs must give the eager bits."""
    g = ci.chung_lu(20_000, exponent=2.1, mean=6.0, seed=3)
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    k, n_s = 40, 296
    om = osamp.sample(g.n, n_s, 4)
    lab = (np.arange(n_s) % k).astype(np.int32)  # every cluster sampled
    omd, labd = torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda()
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM | csc.DEGREE_ORDER) as h:
        csc.csc_profile_reset()
        csc.csc_profile_enable(True)
        l0, f0, i0 = csc.csc_interpolate(h, omd, labd, k, fuzzy=True, max_iter=5000)
        csc.csc_profile_enable(False)
        q = csc.csc_profile_query()
        l1, f1, i1 = csc.csc_interpolate(h, omd, labd, k, fuzzy=True, max_iter=5000)
    assert q.get("cg_compact", {}).get("launches", 0) >= 2  # at least one compaction and the way back
    assert i0.converged and i0.iters == i1.iters
    assert torch.equal(f0, f1) and torch.equal(l0, l1)
    x = f0.cpu().numpy().astype(np.float64)
    b = ointerp.rhs(g.n, om, lab, k)
    res = ointerp.apply_system(lap, ointerp.mask(g.n, om), 1e-3, 4, x) - b
    rres = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    assert np.max(rres) <= 3e-6, rres
    assert np.array_equal(l0.cpu().numpy(), ointerp.labels_from_indicators(f0.cpu().numpy()))


def test_interpolation_compacted_width_shapes():
    """Each width the compaction reaches runs lane groups of that width (the next power of
    two of its 16-byte vectors, one column tile) with a row-range count, thread count and
    form tuned for it and reported like any other tuned shape; a shape pinned for such a
    width is used as it is, and the solve still meets its target."""
    g = ci.chung_lu(20_000, exponent=2.1, mean=6.0, seed=3)
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    k, n_s = 40, 296
    om = osamp.sample(g.n, n_s, 4)
    lab = (np.arange(n_s) % k).astype(np.int32)
    omd, labd = torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda()
    b = ointerp.rhs(g.n, om, lab, k)

    def check(fz):
        x = fz.cpu().numpy().astype(np.float64)
        res = ointerp.apply_system(lap, ointerp.mask(g.n, om), 1e-3, 4, x) - b
        assert np.max(np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)) <= 3e-6

    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM | csc.DEGREE_ORDER) as h:
        _, f0, i0 = csc.csc_interpolate(h, omd, labd, k, fuzzy=True, max_iter=5000)
        narrow = [x for x in csc.csc_graph_tuned_shapes(h) if x["kernel"] == "cg" and x["columns"] < k]
    assert i0.converged and narrow
    check(f0)
    for x in narrow:
        nv = -(-x["columns"] // 4)
        lanes = 2
        while lanes < nv and lanes < 32:
            lanes *= 2
        assert (x["G"], x["NT"], x["tiles"]) == (lanes, 1, 1), x
    w = narrow[0]
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM | csc.DEGREE_ORDER) as h:
        csc.csc_graph_pin_shape(h, "cg", 4, w["columns"], w["G"], 1, 256, 37, 1, 0, 1)
        _, f1, i1 = csc.csc_interpolate(h, omd, labd, k, fuzzy=True, max_iter=5000)
        pinned = [x for x in csc.csc_graph_tuned_shapes(h) if x["kernel"] == "cg" and x["columns"] == w["columns"]]
    assert i1.converged
    assert [(x["G"], x["P"], x["threads"], x["lean"]) for x in pinned] == [(w["G"], 37, 256, 1)]
    check(f1)


# ------------------------------------------- interpolation with g = 1 - h~

def _check_highpass(g, om, lab, k, lam, m, gamma, fz, dense=True):
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    msk = ointerp.mask(g.n, om)
    b = ointerp.rhs(g.n, om, lab, k)
    x = fz.astype(np.float64)
    res = ointerp.apply_highpass(s, msk, gamma, lam, m, x) - b
    rres = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    assert np.max(rres) <= 3e-6
    x_ref, _, _ = ointerp.interpolate_highpass(s, om, lab, k, lam, m, gamma, tol=1e-11)
    if dense:
        lap = olap.laplacian(g.row_ptr, g.col_idx).toarray()
        w, u = np.linalg.eigh(lap)
        a = np.diag(msk) + gamma * (u @ np.diag(1.0 - och.h_tilde(w, lam, m)) @ u.T)
        kappa = np.linalg.cond(a)
        err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
        assert np.all(err <= kappa * rres * (1 + 1e-6) + 1e-9)
    return x_ref


@pytest.mark.parametrize("n_nodes,k,n_s,lam,m,rcm", [(1000, 20, 120, 0.44, 50, False), (1000, 20, 120, 0.44, 50, True),
                                                     (600, 6, 40, 0.3, 20, False)])
def test_interpolation_highpass_matches_oracle(n_nodes, k, n_s, lam, m, rcm):
    g = ci.sbm(n_nodes, k, seed=2)
    om = osamp.sample(g.n, n_s, 2)
    lab = g.labels[om].astype(np.int32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, int(rcm)) as h:
        labels, fz, info = csc.csc_interpolate_highpass(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(),
                                                        k, lam, m, 1e-3, 1e-7, 5000, fuzzy=True)
    assert info.converged and info.max_rel_residual <= 1e-6
    x = fz.cpu().numpy()
    x_ref = _check_highpass(g, om, lab, k, lam, m, 1e-3, x)
    assert np.array_equal(labels.cpu().numpy(), ointerp.labels_from_indicators(x))
    assert oari.ari(labels.cpu().numpy(), ointerp.labels_from_indicators(x_ref)) >= 0.999


def test_interpolation_highpass_cliques():
    g = ci.disjoint_cliques(4, 7)
    om = np.array([0, 9, 15, 27], dtype=np.int64)
    lab = g.labels[om].astype(np.int32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, fz, info = csc.csc_interpolate_highpass(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(),
                                                        4, 0.5, 50, fuzzy=True)
    assert np.array_equal(labels.cpu().numpy(), g.labels)
    assert np.max(np.abs(fz.cpu().numpy() - np.eye(4)[g.labels])) < 2e-3


def test_interpolation_highpass_graph_replay_matches_eager():
    g = ci.sbm(1000, 20, seed=2)
    om = torch.from_numpy(osamp.sample(g.n, 120, 2)).cuda()
    lab = torch.from_numpy(g.labels[om.cpu().numpy()].astype(np.int32)).cuda()
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_profile_enable(True)
        l0, f0, i0 = csc.csc_interpolate_highpass(h, om, lab, 20, 0.44, 50, fuzzy=True)
        csc.csc_profile_enable(False)
        l1, f1, i1 = csc.csc_interpolate_highpass(h, om, lab, 20, 0.44, 50, fuzzy=True)
    assert i0.iters == i1.iters and torch.equal(f0, f1) and torch.equal(l0, l1)


def test_cluster_highpass_recovers_communities():
    """Alg. 2 end to end with g = 1 - h~: ARI against the planted partition, beside L^4."""
    g = ci.sbm(2000, 20, seed=4)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        l4, i4 = csc.csc_cluster(h, 20, seed=1)
        lh, ih = csc.csc_cluster(h, 20, seed=1, flags=csc.HIGHPASS)
    a4 = oari.ari(l4.cpu().numpy(), g.labels)
    ah = oari.ari(lh.cpu().numpy(), g.labels)
    assert ih.cg.converged and ah >= 0.8 and ah >= a4 - 0.05


def test_cluster_highpass_interp_degree():
    """m_interp sets the degree of h~ inside g = 1 - h~ only: a degree-20 regulariser
    still recovers the planted communities, in fewer products than degree 50."""
    g = ci.sbm(2000, 20, seed=4)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        l50, i50 = csc.csc_cluster(h, 20, seed=1, flags=csc.HIGHPASS)
        l20, i20 = csc.csc_cluster(h, 20, seed=1, flags=csc.HIGHPASS, m_interp=20)
    assert i20.cg.converged and i50.cg.converged
    assert i20.lam.lam == i50.lam.lam
    a20 = oari.ari(l20.cpu().numpy(), g.labels)
    assert a20 >= 0.8 and 20 * i20.cg.iters < 50 * i50.cg.iters


def test_check_finite_reports_non_finite_signals():
    """CSC_CHECK_FINITE: a NaN planted on the host in R_in is reported as CSC_E_NUMERIC before
    any filtering; without the flag it flows into Y; a clean block passes and the handle
    stays usable, including csc_cluster with the flag."""
    g = ci.sbm(1000, 20, seed=0)
    r = ci.gaussian_block(g.n, 28, 32, seed=1)
    r[17, 3] = np.nan
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, 0.4, 20, 28, 32, R_in=torch.from_numpy(r).cuda(), flags=0)
        assert torch.isnan(y).any()
        with pytest.raises(csc.CscError) as e:
            csc.csc_filter_random_signals(h, 0.4, 20, 28, 32, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CHECK_FINITE)
        assert e.value.status == nat.CSC_E_NUMERIC
        r[17, 3] = np.inf
        with pytest.raises(csc.CscError) as e:
            csc.csc_filter_random_signals(h, 0.4, 20, 28, 32, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CHECK_FINITE | csc.CLENSHAW)
        assert e.value.status == nat.CSC_E_NUMERIC
        r[17, 3] = 0.5
        y = csc.csc_filter_random_signals(h, 0.4, 20, 28, 32, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CHECK_FINITE | csc.NORMALIZE_ROWS)
        assert torch.isfinite(y).all()
        labels, _ = csc.csc_cluster(h, 20, seed=0, flags=csc.CHECK_FINITE)
        assert oari.ari(labels.cpu().numpy(), g.labels) > 0.8


def test_sampling_wrappers_reject_short_or_mistyped_buffers():
    for fn in (csc.csc_sample, csc.csc_sample_noalloc):
        with pytest.raises(ValueError):
            fn(1000, 120, 0, torch.empty(120, dtype=torch.int32, device="cuda"))
        with pytest.raises(ValueError):
            fn(1000, 120, 0, torch.empty(119, dtype=torch.int64, device="cuda"))
        out = torch.full((121,), -1, dtype=torch.int64, device="cuda")
        fn(1000, 120, 0, out)
        assert torch.equal(out[:120].cpu(), torch.from_numpy(osamp.sample(1000, 120, 0)))
        assert int(out[120]) == -1
