"""The learned lambda_k bracket on the device: features, targets, the network's
forward / gradient / Adam step against the FP64 oracle, the paper-literal
eigencount, and what a trained network gains over the dichotomy without it."""
import math

import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import bracket as obr
from oracle import chebyshev as och
from oracle import laplacian as olap
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


def _params(seed=0):
    rng = np.random.default_rng(seed)
    blocks = {}
    for name, shape in omlp.layout():
        if len(shape) == 2:
            blocks[name] = rng.standard_normal(shape) * math.sqrt(2.0 / shape[0])
        else:
            blocks[name] = rng.standard_normal(shape) * 0.1
    return omlp.pack(blocks).astype(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


# ------------------------------------------------------------ features, targets

@pytest.mark.parametrize("gname", ["sbm", "chung_lu"])
def test_features_match_oracle(gname):
    g = ci.sbm(2000, 10, seed=1) if gname == "sbm" else ci.chung_lu(3000, 2.5, 6.0, seed=1, cutoff=math.sqrt(18000))
    k = 10
    ref = obr.features(g.row_ptr, g.col_idx, k, seed=7)
    for flags in (0, csc.RCM):
        with csc.csc_graph_create(g.row_ptr, g.col_idx, flags) as h:
            f, mu = csc.csc_bracket_features(h, k, seed=7)
        f = f.astype(np.float64)
        assert np.max(np.abs(f[:64] - ref[:64])) <= 2e-5 * abs(ref[0])
        assert np.allclose(mu / g.n, f[:64], rtol=1e-6, atol=0)
        assert f[64] == np.float32(ref[64]) and f[65] == ref[65]
        assert np.array_equal(f[66:], ref[66:].astype(np.float32))


def test_bracket_target_matches_oracle():
    g = ci.sbm(1000, 20, seed=0)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    mu = och.moments(s, och.probe_signals(g.n, 14, 14, seed=3), 50)
    for k in (1, 5, 20, 37):
        lo, hi = csc.csc_bracket_target(mu, k)
        rlo, rhi = obr.target_bracket(mu, k)
        assert abs(lo - rlo) <= 1e-12 and abs(hi - rhi) <= 1e-12


# ------------------------------------------------------------------ network

def test_mlp_init_statistics():
    p = csc.csc_mlp_init(seed=3).cpu().numpy().astype(np.float64)
    blocks = omlp.unpack(p)
    for name, shape in omlp.layout():
        b = blocks[name]
        if len(shape) == 1:
            assert np.all(b == 0)
        else:
            a = math.sqrt(6.0 / shape[0])
            assert np.max(np.abs(b)) <= a and abs(b.mean()) < 0.05 * a
            assert abs(b.std() - a / math.sqrt(3)) < 0.05 * a
    assert np.array_equal(p, csc.csc_mlp_init(seed=3).cpu().numpy())


@pytest.mark.parametrize("B", [1, 37, 300])
def test_mlp_forward_matches_oracle(B):
    p = _params(1)
    x = np.random.default_rng(B).standard_normal((B, 72)).astype(np.float32)
    y = csc.csc_mlp_forward(_dev(p), _dev(x)).cpu().numpy()
    ref, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(y - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("B", [1, 37, 256])
def test_mlp_gradient_matches_oracle(B):
    p = _params(2)
    rng = np.random.default_rng(B + 100)
    x = rng.standard_normal((B, 72)).astype(np.float32)
    t = (rng.standard_normal((B, 2)) * 2.0).astype(np.float32)
    loss, grad = csc.csc_mlp_loss_grad(_dev(p), _dev(x), _dev(t))
    rloss, rgrad = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= 1e-5 * max(1.0, rloss)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - rgrad)) <= 1e-4 * np.max(np.abs(rgrad))
    assert np.linalg.norm(g - rgrad) <= 1e-5 * np.linalg.norm(rgrad)


@pytest.mark.parametrize("t", [1, 7])
def test_adam_step_matches_oracle(t):
    rng = np.random.default_rng(t)
    n = omlp.N_PARAMS
    p, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    m = (rng.standard_normal(n) * 0.1).astype(np.float32)
    v = (rng.random(n) * 0.01).astype(np.float32)
    dp, dm, dv = _dev(p), _dev(m), _dev(v)
    csc.csc_mlp_adam_step(dp, _dev(g), dm, dv, t, 1e-3)
    rp, rm, rv = omlp.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                                v.astype(np.float64), t, 1e-3)
    assert np.allclose(dm.cpu().numpy(), rm, rtol=1e-6, atol=1e-7)
    assert np.allclose(dv.cpu().numpy(), rv, rtol=1e-6, atol=1e-9)
    assert np.max(np.abs(dp.cpu().numpy() - rp)) <= 1e-6 * max(1.0, np.max(np.abs(rp)))


def test_train_full_batch_epochs_match_oracle_adam():
    """Three epochs with batch = n are three full-batch Adam steps of the oracle."""
    n = 48
    rng = np.random.default_rng(9)
    x = rng.standard_normal((n, 72)).astype(np.float32)
    t = rng.standard_normal((n, 2)).astype(np.float32)
    p0 = _params(4)
    dp = _dev(p0)
    hist = csc.csc_mlp_train(dp, _dev(x), _dev(t), 3, n, 1e-3, seed=5)
    p = p0.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for step in range(1, 4):
        loss, g = omlp.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64))
        losses.append(loss)
        p, m, v = omlp.adam_step(p, g, m, v, step, 1e-3)
    assert np.allclose(hist, losses, rtol=1e-5)
    assert np.max(np.abs(dp.cpu().numpy() - p)) <= 2e-5 * np.max(np.abs(p))


# ------------------------------------------------------- paper-literal eigencount

def test_refilter_count_matches_oracle_and_moments():
    g = ci.sbm(1000, 20, seed=0)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    nv, m = 14, 50
    probes = och.probe_signals(g.n, nv, 16, seed=3)
    mu = och.moments(s, probes, m, n_v=nv)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        plain = csc.csc_estimate_lambda_k(h, 20, m, nv, 3)
        lit = csc.csc_estimate_lambda_k_refilter(h, 20, m, nv, 3)
    assert lit.hit and plain.hit
    assert lit.moment_passes == m * lit.iters
    # the count at the answer is the oracle's paper-literal count there, and equals the
    # moments-once count (same probes); both estimators accept the answer
    ref = och.eigencount_refilter(s, probes, lit.lam, m, n_v=nv)
    assert abs(lit.count - ref) <= 1e-4 * 20
    assert abs(lit.count - och.eigencount(mu, lit.lam)) <= 1e-4 * 20
    assert och.round_half_away(ref) == 20
    assert och.round_half_away(och.eigencount(mu, plain.lam)) == 20


# -------------------------------------------------------------- trained network

@pytest.fixture(scope="module")
def trained():
    import multiprocessing as mp

    from csc_inputs.datasets import bracket_graph_arrays
    from paper_1602_02018_gb300 import learned

    n_train, n_test = 480, 120
    tasks = [(i, (2e3, 2e4), (5, 60)) for i in range(n_train + n_test)]
    with mp.get_context("spawn").Pool(8) as pool:
        res = sorted(pool.map(bracket_graph_arrays, tasks, chunksize=8), key=lambda r: r[0])
    graphs = [(ci.CSRGraph(rp, col, lab), k) for _, rp, col, lab, k in res]
    feats, brs = learned.dataset(graphs, m=50, seed=0)
    model = learned.BracketModel.fit(feats[:n_train], brs[:n_train], epochs=300, batch=32, lr=1e-3, seed=0)
    return dict(graphs=graphs, feats=feats, brs=brs, model=model, n_train=n_train)


def test_training_reduces_loss(trained):
    h = trained["model"].loss_history
    assert h.size == 300 and np.all(np.isfinite(h))
    assert h[-1] < 0.2 * h[0]


def test_held_out_coverage(trained):
    nt = trained["n_train"]
    pred = trained["model"].predict_brackets(trained["feats"][nt:])
    br = trained["brs"][nt:]
    cov = (pred[:, 0] <= br[:, 1]) & (pred[:, 1] >= br[:, 0])  # prediction meets the target bracket
    assert cov.mean() >= 0.7
    # narrower than the dichotomy's [0, 2]
    assert np.median(pred[:, 1] - pred[:, 0]) < 0.5


def test_prediction_is_the_bracket_the_estimate_starts_from(trained):
    """csc_bracket_predict gives, from a graph's features, the bracket that
    csc_estimate_lambda_k_learned computes inside for the same graph."""
    nt = trained["n_train"]
    model = trained["model"]
    pred = model.predict_brackets(trained["feats"][nt:nt + 8])
    for i, (g, k) in enumerate(trained["graphs"][nt:nt + 8]):
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
            _, br = model.estimate(h, k, 50, 0, 0)
        assert np.allclose(br, pred[i], rtol=0, atol=1e-9), (br, pred[i])


def test_fit_coverage_rule_meets_its_share(trained):
    """widen_rule "coverage": with the calibrated factor, at least the asked share of the
    held-back samples' predicted intervals meet their target brackets; the fitted and
    held-back split follows val_frac."""
    from paper_1602_02018_gb300 import learned

    nt = trained["n_train"]
    feats, brs = trained["feats"][:nt], trained["brs"][:nt]
    model = learned.BracketModel.fit(feats, brs, epochs=60, batch=32, lr=1e-3, seed=1, coverage=0.8,
                                     widen_rule="coverage")
    assert model.n_val == round(0.15 * nt) and model.n_fit + model.n_val == nt and model.widen >= 1.0
    pred = model.predict_brackets(feats[model.n_fit:])
    br = brs[model.n_fit:]
    cov = (pred[:, 0] <= br[:, 1]) & (pred[:, 1] >= br[:, 0])
    # the interpolated 0.8 quantile of the needed factors lies at or above the
    # floor(0.8 (n - 1)) + 1 smallest of them
    n = len(br)
    assert cov.sum() >= np.floor(0.8 * (n - 1)) + 1
    t = model.predict_targets(feats[model.n_fit:])
    hw = model.widen * np.exp(np.minimum(t[:, 1], 10.0))
    assert np.allclose(pred[:, 0], np.maximum(0.0, t[:, 0] - hw)) and np.allclose(pred[:, 1], np.minimum(2.0, t[:, 0] + hw))


def test_gain_over_the_paper_literal_dichotomy(trained):
    """Paper-literal eigencount: the bracket saves filter passes, and every answer
    is one the unbracketed estimator accepts (round(count) = k)."""
    nt = trained["n_train"]
    model = trained["model"]
    plain_products, learned_products, used = 0, 0, 0
    for g, k in trained["graphs"][nt:]:
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
            a = csc.csc_estimate_lambda_k_refilter(h, k, 50, 0, 0)
            b, _ = model.estimate(h, k, 50, 0, 0, refilter=True)
        plain_products += a.moment_passes
        learned_products += b.moment_passes
        used += b.bracket_used
        assert b.hit == a.hit or not a.hit
        if b.hit:
            assert round(b.count) == k
    assert used >= 0.6 * (len(trained["graphs"]) - nt)
    assert learned_products < 0.8 * plain_products


def test_learned_lambda_gives_the_same_clustering(trained):
    """Moments-once path: CSC labels with the learned lambda_k match the plain
    path's ARI against the planted communities (SBM graphs of the held-out set)."""
    from oracle import ari as oari

    nt = trained["n_train"]
    model = trained["model"]
    diffs = []
    for g, k in trained["graphs"][nt:]:
        if g.labels is None:
            continue
        with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
            a = csc.csc_estimate_lambda_k(h, k, 50, 0, 0)
            b, _ = model.estimate(h, k, 50, 0, 0)
            la, _ = csc.csc_cluster(h, k, lambda_k=a.lam, seed=0)
            lb, _ = csc.csc_cluster(h, k, lambda_k=b.lam, seed=0)
        diffs.append(oari.ari(lb.cpu().numpy(), g.labels) - oari.ari(la.cpu().numpy(), g.labels))
    assert len(diffs) >= 10
    assert abs(float(np.mean(diffs))) <= 0.02
