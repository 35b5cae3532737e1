"""Pins of the oracle's variable-density sampling (Sec. 3.2.3 after Theorem 3.4, the
remark closing Sec. 4.2) and of its weighted decoder."""
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import csc_inputs as ci
from oracle import chebyshev, interp, laplacian, sampling
from oracle.rng import splitmix64_at

TWO64 = 1 << 64


def _ceil_div(a: int, b: int) -> int:
    return -((-a) // b)


# --- the integer inverse CDF ----------------------------------------------------

def test_inverse_cdf_boundaries_exact():
    """The first 64-bit word of each node's range, counted with big integers from
    the cumulative weights, maps to that node and the word before it to the previous one."""
    rng = np.random.default_rng(5)
    q = rng.integers(0, 1 << 32, size=40, dtype=np.uint64)
    q[[3, 4, 17]] = 0  # empty ranges are skipped
    q[-1] = 1
    big_q = int(q.sum())
    cum = np.cumsum([int(v) for v in q])
    first = [_ceil_div(int(c - int(v)) * TWO64, big_q) for c, v in zip(cum, q)]
    prev_pos = None
    words, expect = [], []
    for i, v in enumerate(q):
        if v == 0:
            continue
        words.append(first[i])
        expect.append(i)
        if prev_pos is not None:
            words.append(first[i] - 1)
            expect.append(prev_pos)
        prev_pos = i
    words.append(TWO64 - 1)
    expect.append(len(q) - 1)
    got = sampling.node_of_word(np.array(words, dtype=np.uint64), q)
    assert np.array_equal(got, np.array(expect))
    # each node's share of the 2^64 words is q_i / Q to within one word
    ends = [_ceil_div(int(c) * TWO64, big_q) for c in cum]
    counts = np.diff([0] + ends)
    for i, v in enumerate(q):
        assert abs(Fraction(int(counts[i])) - Fraction(int(v) * TWO64, big_q)) < 1


def test_quantize_bounds():
    rng = np.random.default_rng(1)
    s = rng.exponential(size=500) ** 3
    s[7] = 0.0
    q = sampling.quantize_scores(s)
    assert q.dtype == np.uint64 and int(q.max()) == 1 << 32 and q[7] == 0
    smax = Fraction(float(s.max()))
    for si, qi in zip(s, q):
        exact = Fraction(float(si)) / smax * (1 << 32)
        assert abs(Fraction(int(qi)) - exact) < 1 + Fraction(1, 1 << 19)


@pytest.mark.parametrize("bad", [np.array([1.0, -1e-300]), np.array([np.nan, 1.0]), np.array([np.inf, 1.0]),
                                 np.zeros(4), np.zeros(0)])
def test_invalid_scores(bad):
    with pytest.raises(ValueError):
        sampling.sample_variable_density(bad, 3, 0)


def test_draw_frequencies_follow_weights():
    rng = np.random.default_rng(2)
    s = rng.exponential(size=25) ** 2
    n = 40000
    om, w = sampling.sample_variable_density(s, n, seed=11)
    q = sampling.quantize_scores(s).astype(np.float64)
    expected = n * q / q.sum()
    hits = np.bincount(om, minlength=25)
    chi2 = np.sum((hits - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, 24) > 1e-3
    assert len(om) == n and np.all(np.diff(om) >= 0)
    # every draw of a node carries the same weight Q / (N q_i)
    assert np.allclose(w, (q.sum() / (25 * q[om])).astype(np.float32), rtol=0, atol=0)


def test_flat_profile_is_uniform_with_unit_weights():
    n_nodes, n = 30, 30000
    om, w = sampling.sample_variable_density(np.full(n_nodes, 3.7), n, seed=4)
    assert np.all(w == np.float32(1.0))
    hits = np.bincount(om, minlength=n_nodes)
    expected = n / n_nodes
    chi2 = np.sum((hits - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, n_nodes - 1) > 1e-3


def test_zero_scores_never_drawn_and_single_support():
    s = np.zeros(50)
    s[[4, 20, 21]] = [1.0, 0.5, 2.0]
    om, _ = sampling.sample_variable_density(s, 5000, seed=9)
    assert set(np.unique(om)) <= {4, 20, 21}
    one = np.zeros(12)
    one[6] = 0.25
    om, w = sampling.sample_variable_density(one, 40, seed=1)
    assert np.all(om == 6) and np.all(w == np.float32(1.0 / 12))


def test_power_of_two_rescaling_changes_nothing():
    rng = np.random.default_rng(3)
    s = rng.random(300)
    ref = sampling.sample_variable_density(s, 500, seed=8)
    for e in (-40, -1, 7, 60):
        om, w = sampling.sample_variable_density(np.ldexp(s, e), 500, seed=8)
        assert np.array_equal(om, ref[0]) and np.array_equal(w, ref[1])


def test_seed_is_the_splitmix_stream():
    """Draw t uses SplitMix64 output t: the unsorted draws of n are a prefix of those of n' > n."""
    s = np.arange(1.0, 41.0)
    q = sampling.quantize_scores(s)
    a = sampling.node_of_word(splitmix64_at(13, np.arange(10, dtype=np.uint64)), q)
    b = sampling.node_of_word(splitmix64_at(13, np.arange(30, dtype=np.uint64)), q)
    assert np.array_equal(a, b[:10])
    assert np.array_equal(np.sort(a), sampling.sample_variable_density(s, 10, 13)[0])


def test_scores_estimate_filtered_coherence():
    """E ||(h~(L) R)^T delta_i||^2 = sum_l h~(lambda_l)^2 U_il^2 for R with N(0, 1/d)
    entries; the relative spread per node is sqrt(2/d), that of the sum over nodes
    sqrt(2 sum h~^4 / d) / sum h~^2 (the nodes share the d signals)."""
    g = ci.sbm(80, 4, s=6, seed=2)
    s_mat = laplacian.normalized_adjacency(g.row_ptr, g.col_idx)
    lap = laplacian.dense_laplacian(g.row_ptr, g.col_idx)
    lam_c, m, d = 0.25, 40, 3000
    y = chebyshev.cheb_filter(s_mat, chebyshev.random_signals(80, d, d, seed=6), chebyshev.filter_coeffs(lam_c, m))
    sc = sampling.coherence_scores(y)
    ev, u = np.linalg.eigh(lap)
    expect = (u ** 2) @ (chebyshev.h_tilde(ev, lam_c, m) ** 2)
    rel = np.abs(sc - expect) / expect
    sd = np.sqrt(2.0 / d)
    assert np.max(rel) < 6 * sd
    h = chebyshev.h_tilde(ev, lam_c, m)
    sd_tot = np.sqrt(2.0 * np.sum(h ** 4) / d) / np.sum(h ** 2)
    assert abs(np.sum(sc) / np.sum(expect) - 1.0) < 5 * sd_tot


# --- the weighted decoder ---------------------------------------------------------

def _small_problem(n_nodes=24, k=2, seed=0):
    g = ci.sbm(n_nodes, k, s=5, seed=seed)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    return g, lap


def test_unit_weights_reproduce_eq5():
    g = ci.sbm(200, 4, s=8, seed=1)
    lap = laplacian.laplacian(g.row_ptr, g.col_idx)
    om = sampling.sample(200, 30, seed=2)
    lab = g.labels[om]
    x0, _, _ = interp.interpolate(lap, om, lab, 4, 1e-3, 4, tol=1e-12)
    x1, _, res = interp.interpolate_weighted(lap, om, lab, np.ones(30, np.float32), 4, 1e-3, 4, tol=1e-12)
    assert res < 1e-11
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-8


def test_repeated_draw_equals_doubled_weight():
    g, lap = _small_problem(60, 3, seed=4)
    om = np.array([2, 2, 17, 33, 41, 41, 41, 58])
    lab = g.labels[om]
    w = np.array([0.5, 0.5, 1.25, 2.0, 0.75, 0.75, 0.75, 3.0], np.float32)
    x1, _, _ = interp.interpolate_weighted(lap, om, lab, w, 3, 1e-2, 4, tol=1e-13)
    uo = np.array([2, 17, 33, 41, 58])
    uw = np.array([1.0, 1.25, 2.0, 2.25, 3.0], np.float32)
    x2, _, _ = interp.interpolate_weighted(lap, uo, g.labels[uo], uw, 3, 1e-2, 4, tol=1e-13)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-9


def test_solution_is_the_minimiser_of_the_drawwise_objective():
    g, lap = _small_problem(24, 2, seed=3)
    ld = lap.toarray()
    om = np.array([1, 1, 5, 9, 14, 20, 20])
    lab = np.array([g.labels[i] for i in om])
    lab[5] = 1 - lab[5]  # conflicting observations of node 20 are allowed
    w = np.array([0.5, 0.5, 2.0, 1.0, 0.25, 1.5, 1.0], np.float32)
    gamma, power = 0.05, 2
    x, _, _ = interp.interpolate_weighted(lap, om, lab, w, 2, gamma, power, tol=1e-14)
    f0 = interp.weighted_objective(ld, om, lab, w, gamma, power, x)
    grad0 = interp.weighted_objective(ld, om, lab, w, gamma, power, np.zeros_like(x))
    h = 1e-4
    for i in range(24):
        for j in range(2):
            e = np.zeros_like(x)
            e[i, j] = h
            fd = (interp.weighted_objective(ld, om, lab, w, gamma, power, x + e)[j]
                  - interp.weighted_objective(ld, om, lab, w, gamma, power, x - e)[j]) / (2 * h)
            assert abs(fd) < 1e-6 * max(1.0, grad0[j])
    rng = np.random.default_rng(0)
    for _ in range(20):
        pert = 1e-2 * rng.standard_normal(x.shape)
        assert np.all(interp.weighted_objective(ld, om, lab, w, gamma, power, x + pert) > f0)


def test_common_scale_of_weights_and_gamma_cancels():
    g, lap = _small_problem(60, 3, seed=5)
    om = np.array([3, 8, 8, 25, 44, 51])
    lab = g.labels[om]
    w = np.array([1.0, 0.5, 0.5, 2.0, 1.5, 0.25], np.float32)
    x1, _, _ = interp.interpolate_weighted(lap, om, lab, w, 3, 1e-3, 4, tol=1e-13)
    x2, _, _ = interp.interpolate_weighted(lap, om, lab, w * np.float32(8), 3, 8e-3, 4, tol=1e-13)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-8


def test_pipeline_with_variable_density_recovers_planted_communities():
    """Alg. 2 with variable-density draws and the weighted decoder, end to end in the
    oracle: the planted communities of a small SBM are recovered and the draws carry
    weights Q / (N q) (a sanity check of the wiring; no printed value to pin to)."""
    from oracle import ari, pipeline

    g = ci.sbm(400, 4, s=12.0, seed=7)
    out = pipeline.csc(g.row_ptr, g.col_idx, 4, seed=1, variable_density=True, replicates=5, n=40)
    assert ari.ari(out["labels"], g.labels) >= 0.9
    q = sampling.quantize_scores(sampling.coherence_scores(out["y"]))
    assert np.array_equal(out["weights"], sampling.decoder_weights(q, out["omega"]))
    assert len(out["omega"]) == out["params"]["n"]
