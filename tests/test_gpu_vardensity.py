"""Parity of variable-density sampling (Sec. 3.2.3 after Theorem 3.4), the coherence
scores (remark closing Sec. 4.2) and the weighted decoder with the oracle."""
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


def _gpu_sample(score: np.ndarray, n: int, seed: int):
    idx, w = csc.csc_sample_weighted(torch.from_numpy(score).cuda(), n, seed)
    return idx.cpu().numpy(), w.cpu().numpy()


# ------------------------------------------------------------------ sampling

@pytest.mark.parametrize("kind", ["heavy", "zeros", "flat", "single", "blocks", "tiny"])
@pytest.mark.parametrize("N,n", [(1, 1), (1, 40), (37, 5), (4096, 300), (4097, 3000), (100_003, 2500)])
def test_sample_weighted_bit_exact(kind, N, n):
    score = ci.score_profile(N, kind, seed=N + n)
    idx, w = _gpu_sample(score, n, seed=7)
    ref_idx, ref_w = osamp.sample_variable_density(score, n, 7)
    assert np.array_equal(idx, ref_idx)
    assert np.array_equal(w.view(np.uint32), ref_w.view(np.uint32))


@pytest.mark.parametrize("N,n", [(100_000, 2120), (1_000_000, 922)])
def test_sample_weighted_full_size(N, n):
    """The workload sizes (SBM N = 1e5 with n = 2k ln k for k = 200; Chung-Lu N = 1e6
    with k = 100), scores shaped like coherences (constant per block, 1 / block size)."""
    score = ci.score_profile(N, "blocks", seed=1)
    idx, w = _gpu_sample(score, n, seed=0)
    ref_idx, ref_w = osamp.sample_variable_density(score, n, 0)
    assert np.array_equal(idx, ref_idx)
    assert np.array_equal(w, ref_w)


def test_sample_weighted_more_draws_than_nodes_and_empty():
    score = ci.score_profile(50, "heavy", seed=2)
    idx, w = _gpu_sample(score, 500, seed=3)
    ref_idx, ref_w = osamp.sample_variable_density(score, 500, 3)
    assert np.array_equal(idx, ref_idx) and np.array_equal(w, ref_w)
    idx, w = csc.csc_sample_weighted(torch.from_numpy(score).cuda(), 0, 3)
    assert idx.numel() == 0 and w.numel() == 0


def test_sample_weighted_without_weights_output():
    score = ci.score_profile(999, "zeros", seed=4)
    idx, w = csc.csc_sample_weighted(torch.from_numpy(score).cuda(), 77, 5, weights=False)
    assert w is None
    assert np.array_equal(idx.cpu().numpy(), osamp.sample_variable_density(score, 77, 5)[0])


@pytest.mark.parametrize("bad", ["negative", "nan", "inf", "zero"])
def test_sample_weighted_rejects_bad_scores(bad):
    score = ci.score_profile(5000, "heavy", seed=3)
    if bad == "negative":
        score[17] = -1e-9
    elif bad == "nan":
        score[4999] = np.nan
    elif bad == "inf":
        score[0] = np.inf
    else:
        score[:] = 0.0
    with pytest.raises(csc.CscError):
        csc.csc_sample_weighted(torch.from_numpy(score).cuda(), 100, 0)
    # the library stays usable
    good = ci.score_profile(5000, "heavy", seed=3)
    idx, _ = _gpu_sample(good, 100, 0)
    assert np.array_equal(idx, osamp.sample_variable_density(good, 100, 0)[0])


# ------------------------------------------------------------------ scores

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("N,d,ld", [(1, 1, 8), (1000, 23, 24), (4099, 48, 48), (257, 5, 16)])
def test_coherence_scores_match(dtype, N, d, ld):
    rng = np.random.default_rng(N + d)
    y = rng.standard_normal((N, ld)).astype(dtype)
    y[N // 2] = 0.0  # a zero row keeps score 0 and stays zero
    yt = torch.from_numpy(y).cuda()
    sc = csc.csc_coherence_scores(yt, d).cpu().numpy()
    ref = osamp.coherence_scores(y[:, :d].astype(np.float64))
    assert np.allclose(sc, ref, rtol=1e-13, atol=0)
    assert torch.equal(yt.cpu(), torch.from_numpy(y))  # normalize=False leaves Y alone
    sc2 = csc.csc_coherence_scores(yt, d, normalize=True).cpu().numpy()
    assert np.array_equal(sc2, sc)
    out = yt.cpu().numpy()
    ref_n = och.normalize_rows(y[:, :d].astype(np.float64))
    tol = 1e-6 if dtype == np.float32 else 1e-14
    assert np.allclose(out[:, :d], ref_n, rtol=0, atol=tol)
    assert np.array_equal(out[:, d:], y[:, d:])  # padding columns untouched


@pytest.mark.parametrize("storage", [0, 2])  # F32, F64
def test_filter_then_scores_matches_oracle(storage):
    """Scores of the unnormalised filtered block against the oracle's filter."""
    g = ci.sbm(3000, 10, seed=5)
    d, d_pad, m, lam = 33, 40, 50, 0.3
    r = ci.gaussian_block(g.n, d, d_pad, seed=9)
    s_mat = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    y_ref = och.cheb_filter(s_mat, r[:, :d].astype(np.float64), och.filter_coeffs(lam, m))
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW)
        sc = csc.csc_coherence_scores(y, d).cpu().numpy()
    ref = osamp.coherence_scores(y_ref)
    assert rel(sc, ref) <= (3e-5 if storage == 0 else 1e-11)


# ------------------------------------------------------------------ weighted decoder

def _weighted_case(n_nodes, k, n_draws, seed, kind):
    g = ci.sbm(n_nodes, k, s=12.0, seed=seed)
    score = ci.score_profile(n_nodes, kind, seed=seed)
    om, w = osamp.sample_variable_density(score, n_draws, seed)
    lab = g.labels[om].astype(np.int32)
    return g, om, w, lab


@pytest.mark.parametrize("n_nodes,k,n_draws,power,rcm,kind", [(1000, 20, 200, 4, False, "blocks"),
                                                              (2000, 8, 80, 2, True, "blocks"),
                                                              (777, 7, 700, 4, False, "zeros")])
def test_interpolate_weighted_matches_oracle(n_nodes, k, n_draws, power, rcm, kind):
    g, om, w, lab = _weighted_case(n_nodes, k, n_draws, 3, kind)
    # every cluster needs a draw for a defined indicator; relabel to the clusters drawn
    used = np.unique(lab)
    remap = {c: i for i, c in enumerate(used)}
    lab = np.array([remap[c] for c in lab], dtype=np.int32)
    kk = len(used)
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    x_ref, _, _ = ointerp.interpolate_weighted(lap, om, lab, w, kk, 1e-3, power, tol=1e-11)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM if rcm else 0) as h:
        labels, fz, info = csc.csc_interpolate_weighted(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(),
                                                        torch.from_numpy(w).cuda(), kk, power, 1e-3, 1e-7, 8000,
                                                        fuzzy=True)
    assert info.converged and info.max_rel_residual <= 1e-6
    x = fz.cpu().numpy().astype(np.float64)
    b = ointerp.weighted_rhs(g.n, om, lab, w, kk)
    msk = ointerp.weighted_mask(g.n, om, w)
    res = ointerp.apply_system(lap, msk, 1e-3, power, x) - b
    rres = np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)
    assert np.max(rres) <= 3e-6
    # forward error within cond(A) times the residual
    a = ointerp.system_matrix(lap, msk, 1e-3, power).toarray()
    kappa = np.linalg.cond(a)
    err = np.linalg.norm(x - x_ref, axis=0) / np.linalg.norm(x_ref, axis=0)
    assert np.all(err <= kappa * rres * (1 + 1e-6) + 1e-9)
    assert np.array_equal(labels.cpu().numpy(), ointerp.labels_from_indicators(x))


def test_interpolate_weighted_unit_weights_equal_eq5():
    g = ci.sbm(1000, 20, seed=2)
    om = torch.from_numpy(osamp.sample(g.n, 120, 2)).cuda()
    lab = torch.from_numpy(g.labels[om.cpu().numpy()].astype(np.int32)).cuda()
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        l0, f0, i0 = csc.csc_interpolate(h, om, lab, 20, fuzzy=True)
        l1, f1, i1 = csc.csc_interpolate_weighted(h, om, lab, torch.ones(120, device="cuda"), 20, fuzzy=True)
    assert i0.iters == i1.iters and torch.equal(f0, f1) and torch.equal(l0, l1)
    assert i1.max_rel_residual == pytest.approx(i0.max_rel_residual, rel=1e-12)


def test_interpolate_weighted_repeat_equals_doubled_weight():
    g = ci.sbm(600, 6, s=10.0, seed=4)
    om = np.array([3, 3, 150, 151, 260, 260, 260, 400, 599], dtype=np.int64)
    w = np.array([0.5, 0.5, 1.25, 2.0, 0.75, 0.75, 0.75, 3.0, 1.0], dtype=np.float32)
    uo = np.array([3, 150, 151, 260, 400, 599], dtype=np.int64)
    uw = np.array([1.0, 1.25, 2.0, 2.25, 3.0, 1.0], dtype=np.float32)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        _, f1, _ = csc.csc_interpolate_weighted(h, torch.from_numpy(om).cuda(),
                                                torch.from_numpy(g.labels[om].astype(np.int32)).cuda(),
                                                torch.from_numpy(w).cuda(), 6, fuzzy=True)
        _, f2, _ = csc.csc_interpolate_weighted(h, torch.from_numpy(uo).cuda(),
                                                torch.from_numpy(g.labels[uo].astype(np.int32)).cuda(),
                                                torch.from_numpy(uw).cuda(), 6, fuzzy=True)
    assert torch.equal(f1, f2)


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_interpolate_weighted_rejects_bad_weight(bad):
    g = ci.sbm(100, 5, s=8, seed=2)
    om = torch.tensor([0, 50], dtype=torch.int64, device="cuda")
    lab = torch.tensor([0, 2], dtype=torch.int32, device="cuda")
    w = torch.tensor([1.0, bad], dtype=torch.float32, device="cuda")
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        with pytest.raises(csc.CscError):
            csc.csc_interpolate_weighted(h, om, lab, w, 5)


# ------------------------------------------------------------------ pipeline

@pytest.mark.parametrize("seed", [0, 1])
def test_cluster_vardensity_matches_oracle(seed):
    """csc_cluster with CSC_VARDENSITY against the oracle pipeline with variable density."""
    g = ci.sbm(1000, 20, seed=seed)
    ref = opipe.csc(g.row_ptr, g.col_idx, 20, seed=seed, variable_density=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, info = csc.csc_cluster(h, 20, seed=seed, flags=csc.VARDENSITY)
    lab = labels.cpu().numpy()
    assert info.cg.converged
    assert abs(oari.ari(lab, g.labels) - oari.ari(ref["labels"], g.labels)) <= 0.02
    assert oari.ari(lab, ref["labels"]) >= 0.95


def test_cluster_vardensity_f64_draws_match_oracle():
    """With fp64 storage the scores agree to ~1e-12, so the draws are the oracle's."""
    g = ci.sbm(1000, 20, seed=0)
    ref = opipe.csc(g.row_ptr, g.col_idx, 20, seed=0, variable_density=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, ref["lam"], 50, ref["params"]["d"], ci.signals.pad8(ref["params"]["d"]),
                                          seed=0, storage=csc.F64, flags=csc.CLENSHAW)
        sc = csc.csc_coherence_scores(y, ref["params"]["d"])
        idx, w = csc.csc_sample_weighted(sc, ref["params"]["n"], 0)
    assert np.array_equal(idx.cpu().numpy(), ref["omega"])
    assert np.allclose(w.cpu().numpy(), ref["weights"], rtol=1e-6, atol=0)


def test_cluster_vardensity_helps_on_heterogeneous_sbm():
    """Five communities of 20 nodes beside five of 380, n = 23 draws: the coherence-shaped
    distribution reaches the small communities that uniform sampling mostly misses."""
    sizes = [20] * 5 + [380] * 5
    a_u, a_v = [], []
    for seed in range(6):
        g = ci.sbm(2000, 10, s=16.0, eps=0.02, seed=seed, sizes=sizes)
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
            lu, _ = csc.csc_cluster(h, 10, seed=seed, n=23)
            lv, iv = csc.csc_cluster(h, 10, seed=seed, n=23, flags=csc.VARDENSITY)
        assert iv.cg.converged
        a_u.append(oari.ari(lu.cpu().numpy(), g.labels))
        a_v.append(oari.ari(lv.cpu().numpy(), g.labels))
    assert np.mean(a_v) >= np.mean(a_u) + 0.05


def test_cluster_batched_rejects_vardensity():
    gs = [ci.sbm(200, 4, s=8, seed=i) for i in range(2)]
    with csc.csc_graph_create_batched([(g.row_ptr, g.col_idx) for g in gs]) as h:
        with pytest.raises(csc.CscError):
            csc.csc_cluster_batched(h, [4, 4], flags=csc.VARDENSITY)
