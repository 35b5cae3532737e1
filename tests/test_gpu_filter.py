"""Parity of the Chebyshev path (degrees, Philox signals, Jackson-Chebyshev filter,
row normalisation) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import chebyshev as och
from oracle import laplacian as olap

from .helpers import rel, small_graphs, with_self_loops

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_02018_gb300 import build

    build.build()


GRAPHS = small_graphs()


@pytest.mark.parametrize("name,g", GRAPHS, ids=[n for n, _ in GRAPHS])
@pytest.mark.parametrize("flags", [0, 1])  # 1 = CSC_RCM
def test_degrees_bit_exact(name, g, flags):
    with csc.csc_graph_create(g.row_ptr, g.col_idx, flags | csc.CHECK_SYM) as h:
        deg = csc.csc_graph_degrees(h)
    assert np.array_equal(deg, olap.degrees(g.row_ptr, g.col_idx).astype(np.int32))


def test_self_loops_dropped():
    g = ci.sbm(300, 5, s=8, seed=2)
    rp, cols = with_self_loops(g)
    with csc.csc_graph_create(rp, cols) as h:
        assert h.nnz == g.nnz
        deg = csc.csc_graph_degrees(h)
    assert np.array_equal(deg, olap.degrees(rp, cols).astype(np.int32))


def test_device_input_matches_host_input():
    g = ci.sbm(1000, 20, seed=0)
    with csc.csc_graph_create(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda()) as h:
        assert np.array_equal(csc.csc_graph_degrees(h), np.diff(g.row_ptr).astype(np.int32))


def _oracle_filter(g, r64, lam, m, damped=True, normalize=False):
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    y = och.cheb_filter(s, r64, och.filter_coeffs(lam, m, damped))
    return och.normalize_rows(y) if normalize else y


CASES = [
    # (graph index, d, d_pad, m, lam)
    (6, 28, 32, 50, 0.4375),
    (6, 47, 48, 50, 0.41),
    (6, 56, 56, 100, 0.2),
    (6, 1, 8, 7, 1.2),
    (6, 8, 8, 1, 0.5),
    (6, 13, 16, 2, 0.9),
    (6, 28, 32, 0, 0.6),
    (7, 24, 24, 30, 0.3),
    (0, 4, 8, 10, 0.5),
    (1, 8, 8, 10, 0.5),
    (2, 3, 8, 20, 1.0),
    (3, 17, 24, 33, 0.77),
    (4, 9, 16, 12, 0.25),
    (5, 5, 8, 50, 0.5),
]


@pytest.mark.parametrize("gi,d,d_pad,m,lam", CASES)
@pytest.mark.parametrize("rcm", [0, 1, 8, 9])  # graph flags: none, RCM, degree order, both
@pytest.mark.parametrize("normalize", [False, True])
def test_filter_f32_matches_oracle(gi, d, d_pad, m, lam, rcm, normalize):
    g = GRAPHS[gi][1]
    r = ci.gaussian_block(g.n, d, d_pad, seed=11)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m, normalize=normalize)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, rcm) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.NORMALIZE_ROWS if normalize else 0).cpu().numpy()
    assert y.shape == (g.n, d_pad)
    assert np.all(y[:, d:] == 0)
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("gi,d,d_pad,m,lam", CASES[:6])
def test_filter_f64_matches_oracle(gi, d, d_pad, m, lam):
    g = GRAPHS[gi][1]
    r = ci.gaussian_block(g.n, d, d_pad, seed=5)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=csc.F64, R_in=torch.from_numpy(r).cuda(),
                                          flags=0).cpu().numpy()
    assert y.dtype == np.float64
    assert rel(y, ref) <= 1e-12


@pytest.mark.parametrize("gi,d,d_pad,m,lam", CASES[:6])
def test_filter_bf16_error_bound(gi, d, d_pad, m, lam):
    # bf16 storage (8-bit mantissa) with fp32 arithmetic: each stored X_j carries a
    # relative rounding error <= 2^-9; over m orders of a stable recurrence the
    # error of Y stays within a few percent of ||Y||.
    g = GRAPHS[gi][1]
    r = ci.gaussian_block(g.n, d, d_pad, seed=5)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=csc.BF16, R_in=torch.from_numpy(r).cuda(),
                                          flags=0).cpu().numpy()
    assert rel(y, ref) <= 5e-2


def test_no_jackson_flag():
    g = GRAPHS[6][1]
    r = ci.gaussian_block(g.n, 28, 32, seed=1)
    ref = _oracle_filter(g, r.astype(np.float64), 0.5, 40, damped=False)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, 0.5, 40, 28, 32, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.NO_JACKSON).cpu().numpy()
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("n,d,d_pad,seed", [(1000, 28, 32, 0), (777, 47, 48, 123456789012), (5, 1, 8, 3)])
def test_generated_signals_match_oracle_philox(n, d, d_pad, seed):
    """R drawn on the GPU (Philox + Box-Muller) equals the oracle's draw; m = 0 gives Y = c_0 R."""
    g = ci.erdos_renyi(n, min(1.0, 8.0 / n), seed=1) if n > 5 else ci.path(n)
    c0 = och.filter_coeffs(0.7, 0)[0]
    r_ref = och.random_signals(n, d, d_pad, seed)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        y = csc.csc_filter_random_signals(h, 0.7, 0, d, d_pad, seed=seed, flags=0).cpu().numpy()
    assert np.all(y[:, d:] == 0)
    assert np.max(np.abs(y / c0 - r_ref)) <= 2e-5 * max(1.0, np.max(np.abs(r_ref)))


def test_generated_signals_whole_filter():
    g = GRAPHS[6][1]
    r_ref = och.random_signals(g.n, 28, 32, 42)
    ref = _oracle_filter(g, r_ref, 0.4375, 50, normalize=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, 0.4375, 50, 28, 32, seed=42).cpu().numpy()
    assert rel(y, ref) <= 1e-5


def test_invalid_filter_arguments_have_no_side_effects():
    g = GRAPHS[6][1]
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = torch.full((g.n, 32), 7.0, device="cuda")
        for args in [(0.5, 10, 28, 30), (0.5, 10, 40, 32), (2.5, 10, 28, 32), (0.5, -1, 28, 32)]:
            with pytest.raises(csc.CscError):
                csc.csc_filter_random_signals(h, *args, Y_out=y)
        assert torch.all(y == 7.0)


def test_filter_full_size_sbm_1e5():
    """Full-size SBM (N = 1e5, k = 200, d = 47 -> 48, m = 50) in the benchmark's launch configuration."""
    g = ci.sbm(100_000, 200, seed=0)
    r = ci.gaussian_block(g.n, 47, 48, seed=0)
    ref = _oracle_filter(g, r.astype(np.float64), 0.40625, 50, normalize=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        y = csc.csc_filter_random_signals(h, 0.40625, 50, 47, 48, R_in=torch.from_numpy(r).cuda()).cpu().numpy()
    assert rel(y, ref) <= 1e-5


SHAPES = [(2, 1), (2, 2), (2, 3), (4, 1), (4, 2), (4, 3), (8, 1), (8, 2), (8, 3), (16, 1), (16, 2), (32, 1),
          (32, 2)]


@pytest.mark.parametrize("G,NT", SHAPES)
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("global_index", [0, 1])
def test_every_compiled_shape_f32(G, NT, threads, global_index):
    """Each compiled (lanes per row, vectors per lane) pair and CTA size gives the oracle's
    filter (ragged row ranges: P = 37)."""
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 47, 48, 20, 0.43
    tiles = -(-(d_pad // 4) // (G * NT))
    r = ci.gaussian_block(g.n, d, d_pad, seed=3)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        csc.csc_graph_pin_shape(h, "cheb_step", 4, d_pad, G, NT, threads, 37, tiles, global_index)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(), flags=0).cpu().numpy()
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("G,NT", [(2, 3), (8, 1), (4, 2), (16, 1)])
@pytest.mark.parametrize("storage,tol", [(1, 5e-2), (2, 1e-12)])
def test_shapes_bf16_f64(G, NT, storage, tol):
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 28, 32, 15, 0.5
    vec = 8 if storage == 1 else 2
    tiles = -(-(d_pad // vec) // (G * NT))
    r = ci.gaussian_block(g.n, d, d_pad, seed=4)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_graph_pin_shape(h, "cheb_step", 2 if storage == 1 else 8, d_pad, G, NT, 256, 29, tiles)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=0).cpu().numpy()
    assert rel(y, ref) <= tol


def test_pin_shape_rejects_bad_shapes():
    g = GRAPHS[6][1]
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cheb_step", 4, 48, 4, 3, 384, 10, 1, 0)   # threads
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cheb_step", 4, 48, 4, 1, 256, 10, 1, 0)   # tiles
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cg", 4, 200, 32, 2, 256, 10, 1, -1)       # index source 0 or 1
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cheb_step", 4, 48, 4, 3, 256, 10, 1, 2)    # index source 0 or 1
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cheb_step", 4, 48, 4, 3, 256, 10, 1, 0, 1)  # lean: Clenshaw and CG only
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "clenshaw", 4, 48, 4, 3, 256, 10, 1, 0, 1)   # lean: NT = 1 only
        with pytest.raises(csc.CscError):
            csc.csc_graph_pin_shape(h, "cg", 4, 48, 16, 1, 512, 10, 1, 0, 1)        # lean: 256 threads only


def test_graph_replay_matches_eager_launches():
    """Without per-launch timing the m orders replay a captured CUDA graph; the result
    is bit-identical to the eager launches, and every replayed kernel is counted."""
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 47, 48, 30, 0.43
    r = torch.from_numpy(ci.gaussian_block(g.n, d, d_pad, seed=3)).cuda()
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_profile_enable(True)
        eager = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=r, flags=0).clone()
        csc.csc_profile_enable(False)
        csc.csc_profile_reset()
        first = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=r, flags=0).clone()
        n1 = csc.csc_profile_launches()
        second = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=r, flags=0).clone()
        n2 = csc.csc_profile_launches() - n1
        other = csc.csc_filter_random_signals(h, 0.9, m, d, d_pad, R_in=r, flags=0).clone()
    torch.cuda.synchronize()
    assert torch.equal(eager, first) and torch.equal(first, second)
    assert n1 == n2 >= m + 1  # copy-in + m orders (+ heavy-row launches, if any)
    ref = _oracle_filter(g, r.cpu().numpy().astype(np.float64), 0.9, m)
    assert rel(other.cpu().numpy(), ref) <= 1e-5  # new coefficients reach the replay


# ----------------------------------------------------- Clenshaw evaluation

@pytest.mark.parametrize("gi,d,d_pad,m,lam", CASES)
@pytest.mark.parametrize("rcm", [0, 1, 8, 9])  # graph flags: none, RCM, degree order, both
@pytest.mark.parametrize("normalize", [False, True])
def test_clenshaw_f32_matches_oracle(gi, d, d_pad, m, lam, rcm, normalize):
    """Clenshaw's backward recurrence gives the oracle's forward-recurrence features."""
    g = GRAPHS[gi][1]
    r = ci.gaussian_block(g.n, d, d_pad, seed=11)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m, normalize=normalize)
    flags = csc.CLENSHAW | (csc.NORMALIZE_ROWS if normalize else 0)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, rcm) as h:
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(),
                                          flags=flags).cpu().numpy()
    assert np.all(y[:, d:] == 0)
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("n,d,d_pad,seed", [(1000, 28, 32, 0), (777, 47, 48, 123456789012), (5, 1, 8, 3)])
@pytest.mark.parametrize("m", [1, 2, 30])
def test_clenshaw_regenerated_signals_match_oracle(n, d, d_pad, seed, m):
    """R regenerated from Philox in every order equals the oracle's draw of the block."""
    g = ci.erdos_renyi(n, min(1.0, 8.0 / n), seed=1) if n > 5 else ci.path(n)
    r_ref = och.random_signals(n, d, d_pad, seed)
    ref = _oracle_filter(g, r_ref, 0.7, m, normalize=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        y = csc.csc_filter_random_signals(h, 0.7, m, d, d_pad, seed=seed,
                                          flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).cpu().numpy()
    assert rel(y, ref) <= 2e-5


@pytest.mark.parametrize("G,NT", SHAPES)
@pytest.mark.parametrize("threads", [256, 512])
@pytest.mark.parametrize("global_index", [0, 1])
def test_clenshaw_every_compiled_shape(G, NT, threads, global_index):
    """Each (lanes, vectors) pair and CTA size; rows normalised in the last order when one
    tile holds a row, by the separate pass otherwise."""
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 47, 48, 20, 0.43
    tiles = -(-(d_pad // 4) // (G * NT))
    r = ci.gaussian_block(g.n, d, d_pad, seed=3)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m, normalize=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        csc.csc_graph_pin_shape(h, "clenshaw", 4, d_pad, G, NT, threads, 37, tiles, global_index)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).cpu().numpy()
    assert rel(y, ref) <= 1e-5


@pytest.mark.parametrize("G", [2, 4, 8, 16, 32])
@pytest.mark.parametrize("global_index", [0, 1])
@pytest.mark.parametrize("storage,tol", [(0, 1e-5), (1, 5e-2)])
def test_clenshaw_lean_form(G, global_index, storage, tol):
    """The lean form (at most 4 neighbour rows in flight per lane, 5 CTAs of 256 threads per
    SM) of every one-vector shape, both index sources, fp32 and bf16 storage; the tuned-shape
    report gives the pinned variant back."""
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 47, 48, 20, 0.43
    vec = 8 if storage == 1 else 4
    tiles = -(-(d_pad // vec) // G)
    r = ci.gaussian_block(g.n, d, d_pad, seed=3)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m, normalize=True)
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        csc.csc_graph_pin_shape(h, "clenshaw", 2 if storage == 1 else 4, d_pad, G, 1, 256, 37, tiles, global_index,
                                lean=1)
        shapes = csc.csc_graph_tuned_shapes(h)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).cpu().numpy()
    assert [x["lean"] for x in shapes] == [1] and shapes[0]["global_index"] == global_index
    assert rel(y, ref) <= tol


@pytest.mark.parametrize("storage,tol", [(1, 5e-2), (2, 1e-12)])
@pytest.mark.parametrize("G,NT", [(2, 3), (8, 1), (4, 2)])
def test_clenshaw_bf16_f64(storage, tol, G, NT):
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 28, 32, 15, 0.5
    vec = 8 if storage == 1 else 2
    tiles = -(-(d_pad // vec) // (G * NT))
    r = ci.gaussian_block(g.n, d, d_pad, seed=4)
    ref = _oracle_filter(g, r.astype(np.float64), lam, m)
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_graph_pin_shape(h, "clenshaw", 2 if storage == 1 else 8, d_pad, G, NT, 256, 29, tiles, 0)
        y = csc.csc_filter_random_signals(h, lam, m, d, d_pad, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW).cpu().numpy()
    assert rel(y, ref) <= tol


def test_clenshaw_graph_replay_matches_eager():
    g = GRAPHS[6][1]
    d, d_pad, m, lam = 47, 48, 30, 0.43
    with csc.csc_graph_create(g.row_ptr, g.col_idx) as h:
        csc.csc_profile_enable(True)
        eager = csc.csc_filter_random_signals(h, lam, m, d, d_pad, seed=5,
                                              flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).clone()
        csc.csc_profile_enable(False)
        a = csc.csc_filter_random_signals(h, lam, m, d, d_pad, seed=5, flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).clone()
        b = csc.csc_filter_random_signals(h, lam, m, d, d_pad, seed=5, flags=csc.CLENSHAW | csc.NORMALIZE_ROWS).clone()
        fwd = csc.csc_filter_random_signals(h, lam, m, d, d_pad, seed=5, flags=csc.NORMALIZE_ROWS).clone()
    torch.cuda.synchronize()
    assert torch.equal(eager, a) and torch.equal(a, b)
    assert rel(a.cpu().numpy(), fwd.cpu().numpy()) <= 1e-5
