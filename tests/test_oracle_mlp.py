"""Pins of the bracket-regressor oracle (oracle/mlp.py) and its features and targets
(oracle/bracket.py) against values fixed by the mathematics."""
import math

import numpy as np

import csc_inputs as ci
from oracle import bracket as obr
from oracle import chebyshev as och
from oracle import laplacian as olap
from oracle import mlp as omlp


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    blocks = {}
    for name, shape in omlp.layout():
        fan_in = shape[0] if len(shape) == 2 else 1
        blocks[name] = rng.standard_normal(shape) * scale * (math.sqrt(2.0 / fan_in) if len(shape) == 2 else 0.1)
    return omlp.pack(blocks)


def test_parameter_count():
    assert omlp.N_PARAMS == 72 * 256 + 256 + 256 * 256 + 256 + 256 * 2 + 2 == 84994


def test_smooth_l1_hand_values():
    # e = 0.5 -> 0.125, e = 2 -> 1.5, e = -3 -> 2.5, e = 0 -> 0 ; mean of the four
    y = np.array([[0.5, 2.0], [-3.0, 0.0]])
    assert omlp.smooth_l1(y, np.zeros_like(y)) == (0.125 + 1.5 + 2.5 + 0.0) / 4


def test_hand_set_network():
    """W1 passes inputs 0 and 1 (and their negatives) through; W2 is an identity on
    those four units; W3 recombines them: Y = (x0 + 2, x1 - 3) for any x."""
    b = {name: np.zeros(shape) for name, shape in omlp.layout()}
    b["W1"][0, 0], b["W1"][0, 1], b["W1"][1, 2], b["W1"][1, 3] = 1.0, -1.0, 1.0, -1.0
    for u in range(4):
        b["W2"][u, u] = 1.0
    b["W3"][0, 0], b["W3"][1, 0], b["W3"][2, 1], b["W3"][3, 1] = 1.0, -1.0, 1.0, -1.0
    b["b3"][:] = [2.0, -3.0]
    x = np.random.default_rng(1).standard_normal((9, 72))
    y, _ = omlp.forward(omlp.pack(b), x)
    assert np.allclose(y, np.stack([x[:, 0] + 2.0, x[:, 1] - 3.0], axis=1), atol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = _params(3)
    x = rng.standard_normal((6, 72))
    t = rng.standard_normal((6, 2)) * 2.0  # both smooth-L1 branches occur
    _, g = omlp.loss_and_grad(p, x, t)
    # every W3/b3 entry plus a random subset of the rest
    n3 = 256 * 2 + 2
    idx = np.concatenate([np.arange(omlp.N_PARAMS - n3, omlp.N_PARAMS),
                          rng.choice(omlp.N_PARAMS - n3, 300, replace=False)])
    h = 1e-6
    fd = np.empty(idx.size)
    for q, i in enumerate(idx):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd[q] = (omlp.smooth_l1(omlp.forward(pp, x)[0], t) - omlp.smooth_l1(omlp.forward(pm, x)[0], t)) / (2 * h)
    err = np.abs(fd - g[idx])
    assert np.max(err) <= 1e-7 * max(1.0, np.max(np.abs(g[idx])))
    assert np.count_nonzero(g[idx]) > idx.size // 4  # not a vacuous comparison


def test_first_adam_step_is_signed_lr():
    rng = np.random.default_rng(5)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    z = np.zeros(100)
    p1, m1, v1 = omlp.adam_step(p, g, z, z, 1, 1e-3)
    assert np.allclose(p1 - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_converges_on_a_quadratic():
    """Adam on f(p) = |p - c|^2 / 2 (gradient p - c) reaches c."""
    c = np.array([1.0, -2.0, 0.5])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        p, m, v = omlp.adam_step(p, p - c, m, v, t, 1e-2)
    assert np.max(np.abs(p - c)) < 1e-3


def test_degree_quantiles_lower_rule():
    rng = np.random.default_rng(2)
    for n in (1, 2, 7, 100, 1001):
        deg = rng.integers(0, 50, n)
        assert np.array_equal(obr.degree_quantiles(deg), np.quantile(deg, obr.QUANTILES, method="lower"))


def test_feature_layout():
    g = ci.sbm(600, 6, seed=1)
    f = obr.features(g.row_ptr, g.col_idx, 6, seed=3)
    assert f.shape == (72,)
    assert f[64] == math.log(600) and f[65] == 6
    assert np.allclose(f[66:], np.log1p(obr.degree_quantiles(np.diff(g.row_ptr))))
    # mu_0 / N is the mean squared probe entry, close to 1
    assert abs(f[0] - 1.0) < 0.1
    # |mu_j| <= mu_0 since |T_j| <= 1 on the spectrum
    assert np.all(np.abs(f[:64]) <= f[0] * (1 + 1e-12))


def test_bracket_on_cliques_lies_in_the_gap():
    """k disjoint K_s: spectrum 0 (x k), s/(s-1) (x k(s-1)).  With every basis vector
    as a probe the count is exact, and k +- 1/2 are crossed inside (0, s/(s-1))."""
    k, s = 4, 7
    g = ci.disjoint_cliques(k, s)
    sm = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    mu = och.moments(sm, np.eye(g.n), 50, n_v=1)
    lo, hi = obr.target_bracket(mu, k)
    assert 0.0 < lo < hi < s / (s - 1)
    assert abs(och.eigencount(mu, lo) - (k - 0.5)) < 1e-9
    assert abs(och.eigencount(mu, hi) - (k + 0.5)) < 1e-9


def test_count_is_nondecreasing_in_lambda():
    g = ci.chung_lu(3000, exponent=2.5, mean=6.0, seed=2, cutoff=math.sqrt(6.0 * 3000))
    sm = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    mu = och.moments(sm, och.probe_signals(g.n, 8, 8, 1), 50)
    c = np.array([och.eigencount(mu, lam) for lam in np.linspace(0, 2, 2001)])
    assert np.all(np.diff(c) >= -1e-9 * g.n)


def test_target_roundtrip():
    t = obr.bracket_to_target(0.2, 0.3)
    lo, hi = obr.target_to_bracket(t)
    assert abs(lo - 0.2) < 1e-15 and abs(hi - 0.3) < 1e-15
    lo2, hi2 = obr.target_to_bracket(t, widen=100.0)
    assert lo2 == 0.0 and hi2 == 2.0
