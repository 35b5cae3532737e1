"""Parity on graphs with hub rows (degree above the 256-edge threshold): the filter,
the moments and the interpolation split such rows off to one CTA each, and their
results must not depend on that split."""
import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import chebyshev as och
from oracle import interp as ointerp
from oracle import laplacian as olap
from oracle import sampling as osamp

from .helpers import rel

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


def hub_graph(n=3000, k=10, seed=0):
    """SBM plus four hubs of degree exactly 257, 256 (the threshold), 1000 and n - 1."""
    base = ci.sbm(n, k, s=12.0, seed=seed)
    nbrs = [set(base.col_idx[base.row_ptr[v]:base.row_ptr[v + 1]].tolist()) for v in range(n)]
    rng = np.random.default_rng(seed + 1)
    for hub, deg in [(3, n - 1), (2, 1000), (1, 256), (0, 257)]:  # later hubs see earlier hubs' edges
        free = np.array(sorted(set(range(n)) - nbrs[hub] - {hub}), dtype=np.int64)
        for v in rng.choice(free, size=deg - len(nbrs[hub]), replace=False).tolist():
            nbrs[hub].add(v)
            nbrs[v].add(hub)
    i = np.concatenate([np.full(len(nb), v) for v, nb in enumerate(nbrs)])
    j = np.concatenate([np.array(sorted(nb), dtype=np.int64) for nb in nbrs])
    return ci.from_edges(n, i, j, labels=base.labels)


HUB = hub_graph()
POWER_LAW = ci.chung_lu(20_000, exponent=2.1, mean=6.0, seed=4)


def test_graphs_have_heavy_rows():
    deg = np.diff(HUB.row_ptr)
    assert list(deg[:4]) == [257, 256, 1000, HUB.n - 1]
    assert np.sum(np.diff(POWER_LAW.row_ptr) > 256) >= 5


def _oracle_filter(g, r64, lam, m):
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    return och.cheb_filter(s, r64, och.filter_coeffs(lam, m))


@pytest.mark.parametrize("gname", ["hub", "power_law"])
@pytest.mark.parametrize("rcm", [0, 1, 8, 9])  # graph flags: none, RCM, degree order, both
def test_filter_f32_heavy(gname, rcm):
    g = HUB if gname == "hub" else POWER_LAW
    d, d_pad, m, lam = 21, 24, 40, 0.3
    r = ci.gaussian_block(g.n, d, d_pad, seed=9)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, rcm) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=0).cpu().numpy()
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("G,NT,threads", [(2, 1, 256), (4, 3, 512), (8, 2, 256), (32, 1, 512), (32, 2, 256)])
def test_filter_pinned_shapes_heavy(G, NT, threads):
    """Heavy rows under each lane layout, including several column tiles."""
    g = HUB
    d, d_pad, m, lam = 47, 48, 20, 0.43
    tiles = -(-(d_pad // 4) // (G * NT))
    r = ci.gaussian_block(g.n, d, d_pad, seed=3)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_graph_pin_shape(h, "cheb_step", 4, d_pad, G, NT, threads, 41, tiles, 0)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=0).cpu().numpy()
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("gname", ["hub", "power_law"])
@pytest.mark.parametrize("G", [2, 8, 16, 32])
@pytest.mark.parametrize("storage,tol", [(0, 1e-5), (1, 5e-2)])
def test_clenshaw_lean_heavy(gname, G, storage, tol):
    """The lean Clenshaw form's row ranges beside the heavy-row launch, on graphs with hubs:
    every order (the first, the middle ones, the last with its normalisation) against the
    oracle, in fp32 and bf16 storage."""
    g = HUB if gname == "hub" else POWER_LAW
    d, d_pad, m, lam = 47, 48, 20, 0.43
    vec = 8 if storage == 1 else 4
    tiles = -(-(d_pad // vec) // G)
    r = ci.gaussian_block(g.n, d, d_pad, seed=3)
    ref = och.normalize_rows(_oracle_filter(g, r.astype(np.float64), lam, m))
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM | csc.DEGREE_ORDER) as h:
        csc.csc_graph_pin_shape(h, "clenshaw", 2 if storage == 1 else 4, d_pad, G, 1, 256, 41, tiles, 0, lean=1)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).cpu().numpy()
    assert rel(y, ref) <= tol


@pytest.mark.parametrize("storage,tol", [(1, 5e-2), (2, 1e-12)])
def test_filter_bf16_f64_heavy(storage, tol):
    g = POWER_LAW
    d, d_pad, m, lam = 28, 32, 30, 0.5
    r = ci.gaussian_block(g.n, d, d_pad, seed=4)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=0).cpu().numpy()
    assert rel(y, ref) <= tol


@pytest.mark.parametrize("gname", ["hub", "power_law"])
def test_moments_heavy(gname):
    g = HUB if gname == "hub" else POWER_LAW
    n_mom, n_v = 41, 12
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    ref = och.moments(s, och.probe_signals(g.n, n_v, n_v, seed=5), n_mom - 1)[:n_mom]
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        mu = csc.csc_kpm_moments(h, n_mom, n_v, seed=5)
        mu_bf = csc.csc_kpm_moments(h, n_mom, n_v, seed=5, storage=csc.BF16)
    assert np.max(np.abs(mu - ref)) <= 2e-5 * abs(ref[0])
    assert np.max(np.abs(mu_bf - ref)) <= 2e-2 * abs(ref[0])


@pytest.mark.parametrize("power", [1, 2, 4])
@pytest.mark.parametrize("G,NT,threads,lean", [(2, 1, 256, 0), (8, 1, 512, 0), (32, 2, 256, 0), (8, 1, 256, 1)])
def test_interpolation_heavy(power, G, NT, threads, lean):
    """CG on the hub graph: the first product of the chain (weighted) and the fused
    A p product both take the heavy-row path; <p, A p> sums their partials."""
    g = HUB
    k, ld = 10, 12
    lap = olap.laplacian(g.row_ptr, g.col_idx)
    om = osamp.sample(g.n, 300, 7)
    lab = g.labels[om].astype(np.int32)
    x_ref, _, _ = ointerp.interpolate(lap, om, lab, k, 1e-3, power, tol=1e-11)
    tiles = -(-(ld // 4) // (G * NT))
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_graph_pin_shape(h, "cg", 4, ld, G, NT, threads, 19, tiles, 0, lean)
        labels, fz, info = csc.csc_interpolate(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(), k,
                                               power, 1e-3, 1e-7, 5000, fuzzy=True)
    assert info.converged and info.max_rel_residual <= 1e-6
    x = fz.cpu().numpy()
    b = ointerp.rhs(g.n, om, lab, k)
    msk = ointerp.mask(g.n, om)
    res = ointerp.apply_system(lap, msk, 1e-3, power, x.astype(np.float64)) - b
    assert np.max(np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)) <= 3e-6
    assert rel(x, x_ref) <= 1e-3
    assert np.array_equal(labels.cpu().numpy(), ointerp.labels_from_indicators(x))


@pytest.mark.parametrize("gname", ["hub", "power_law"])
@pytest.mark.parametrize("normalize", [False, True])
def test_clenshaw_heavy(gname, normalize):
    g = HUB if gname == "hub" else POWER_LAW
    d, d_pad, m, lam = 21, 24, 40, 0.3
    r = ci.gaussian_block(g.n, d, d_pad, seed=9)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    if normalize:
        ref = och.normalize_rows(ref)
    flags = csc.CLENSHAW | (csc.NORMALIZE_ROWS if normalize else 0)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=flags)
    assert rel(y.cpu().numpy(), ref) <= 1e-5


def test_interpolation_highpass_heavy():
    g = HUB
    k = 10
    om = osamp.sample(g.n, 300, 7)
    lab = g.labels[om].astype(np.int32)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        labels, fz, info = csc.csc_interpolate_highpass(h, torch.from_numpy(om).cuda(), torch.from_numpy(lab).cuda(),
                                                        k, 0.35, 40, 1e-3, 1e-7, 5000, fuzzy=True)
    assert info.converged
    x = fz.cpu().numpy().astype(np.float64)
    b = ointerp.rhs(g.n, om, lab, k)
    res = ointerp.apply_highpass(s, ointerp.mask(g.n, om), 1e-3, 0.35, 40, x) - b
    assert np.max(np.linalg.norm(res, axis=0) / np.linalg.norm(b, axis=0)) <= 3e-6
    assert np.array_equal(labels.cpu().numpy(), ointerp.labels_from_indicators(x))
