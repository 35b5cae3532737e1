"""Textbook spectra pin the oracle's normalized Laplacian (Sec. 2.1)."""
import numpy as np
import pytest

import csc_inputs as ci
from oracle import laplacian


def spectrum(g):
    return np.sort(np.linalg.eigvalsh(laplacian.dense_laplacian(g.row_ptr, g.col_idx)))


def test_disjoint_cliques():
    k, s = 4, 6
    ev = spectrum(ci.disjoint_cliques(k, s))
    expect = np.sort(np.concatenate([np.zeros(k), np.full(k * (s - 1), s / (s - 1))]))
    assert np.allclose(ev, expect, atol=1e-12)


@pytest.mark.parametrize("n", [5, 8, 13])
def test_cycle(n):
    ev = spectrum(ci.ring(n))
    expect = np.sort(1 - np.cos(2 * np.pi * np.arange(n) / n))
    assert np.allclose(ev, expect, atol=1e-12)


def test_complete():
    n = 9
    ev = spectrum(ci.complete(n))
    expect = np.concatenate([[0.0], np.full(n - 1, n / (n - 1))])
    assert np.allclose(ev, expect, atol=1e-12)


def test_complete_bipartite_reaches_two():
    a, b = 3, 5
    ev = spectrum(ci.complete_bipartite(a, b))
    expect = np.concatenate([[0.0], np.ones(a + b - 2), [2.0]])
    assert np.allclose(ev, expect, atol=1e-12)


@pytest.mark.parametrize("n", [2, 6, 11])
def test_path(n):
    ev = spectrum(ci.path(n))
    expect = np.sort(1 - np.cos(np.pi * np.arange(n) / (n - 1)))
    assert np.allclose(ev, expect, atol=1e-12)


def test_bounds_on_random_graph():
    g = ci.sbm(200, 4, s=8, seed=3)
    ev = spectrum(g)
    assert ev[0] > -1e-12 and ev[-1] < 2 + 1e-12
    assert abs(ev[0]) < 1e-12


def test_degrees_drop_self_loops_and_isolated_node():
    # 0-1, 1-2, self loop on 2, node 3 isolated
    rp = np.array([0, 1, 3, 5, 5], dtype=np.int64)
    ci_ = np.array([1, 0, 2, 1, 2], dtype=np.int32)
    deg = laplacian.degrees(rp, ci_)
    assert np.array_equal(deg, [1, 2, 1, 0])
    lap = laplacian.dense_laplacian(rp, ci_)
    assert lap[3, 3] == 1.0 and np.all(lap[3, :3] == 0)
    assert lap[2, 2] == 1.0  # self loop excluded from D and from W
    assert np.isclose(lap[0, 1], -1 / np.sqrt(2))
