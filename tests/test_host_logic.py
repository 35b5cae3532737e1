"""Host-side logic of libcsc checked on the CPU: CSR validation errors, the
Jackson-Chebyshev coefficients and the eigencount, against the oracle."""
import ctypes

import numpy as np
import pytest

import csc_inputs as ci
from oracle import chebyshev as och


@pytest.fixture(scope="module")
def L():
    from paper_1602_02018_gb300 import _native, build

    build.build()
    return _native


def _create(nat, rp, colidx, flags=0):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    out = ctypes.c_void_p()
    st = nat.lib().csc_graph_create(len(rp) - 1, len(colidx), rp.ctypes.data_as(ctypes.c_void_p),
                                    colidx.ctypes.data_as(ctypes.c_void_p), None, flags, None, ctypes.byref(out))
    return st, out


@pytest.mark.parametrize("rp,cols,flags", [
    ([1, 1, 2], [0, 1], 0),             # row_ptr[0] != 0
    ([0, 1, 3], [1, 0], 0),             # row_ptr[N] != nnz
    ([0, 2, 2], [1, 0], 0),             # unsorted row
    ([0, 2, 3], [1, 1, 0], 0),          # duplicate column
    ([0, 1, 2], [5, 0], 0),             # out of range
    ([0, 1, 1], [1], 2),                # asymmetric with CSC_CHECK_SYM
])
def test_malformed_csr_rejected(L, rp, cols, flags):
    st, h = _create(L, rp, cols, flags)
    assert st == L.CSC_E_CSR
    assert not h.value
    assert len(L.lib().csc_last_error()) > 0


def _ring(n, k):
    """Circulant graph: node i joined to i +- 1..k (mod n), rows sorted."""
    cols = np.sort((np.arange(n)[:, None] + np.r_[-k:0, 1:k + 1][None, :]) % n, axis=1)
    return np.arange(0, 2 * k * n + 1, 2 * k, dtype=np.int64), cols.astype(np.int32).ravel()


@pytest.mark.parametrize("flags", [0, 2])
def test_malformed_large_csr_reports_first_bad_row(L, flags):
    """A CSR large enough to be checked by several host threads: with faults planted in a
    late and an early row (and, with CSC_CHECK_SYM, asymmetric rows), the message names
    the earliest fault, as a row-by-row scan would."""
    n, k = 300_000, 3
    rp, cols = _ring(n, k)
    late, early = 250_123, 40_007
    for row in (late, early):
        a = rp[row]
        cols[a], cols[a + 1] = cols[a + 1], cols[a]  # unsorted row
    st, h = _create(L, rp, cols, flags)
    assert st == L.CSC_E_CSR and not h.value
    msg = L.lib().csc_last_error().decode()
    assert f"row {early} not strictly increasing" in msg, msg
    if flags:
        rp, cols = _ring(n, k)
        for row in (late, early):
            cols[rp[row] + 2 * k - 1] = (row + k + 1) % n  # (row, row + k) -> (row, row + k + 1), still sorted
        st, h = _create(L, rp, cols, flags)
        assert st == L.CSC_E_CSR and not h.value
        msg = L.lib().csc_last_error().decode()
        assert msg.startswith(f"matrix not symmetric: ({early}, {early + k + 1}) present"), msg


def test_invalid_arguments(L):
    out = ctypes.c_void_p()
    assert L.lib().csc_graph_create(0, 0, None, None, None, 0, None, ctypes.byref(out)) == L.CSC_E_INVALID
    rp = np.array([0, 0], np.int64)
    w = np.ones(1, np.float32)
    assert L.lib().csc_graph_create(1, 0, rp.ctypes.data_as(ctypes.c_void_p), None,
                                    w.ctypes.data_as(ctypes.c_void_p), 0, None,
                                    ctypes.byref(out)) == L.CSC_E_UNSUPPORTED
    c = np.empty(4)
    assert L.lib().csc_chebyshev_coefficients(2.5, 3, 0, c.ctypes.data_as(ctypes.c_void_p)) == L.CSC_E_INVALID
    assert L.lib().csc_chebyshev_coefficients(0.5, -1, 0, c.ctypes.data_as(ctypes.c_void_p)) == L.CSC_E_INVALID
    assert L.lib().csc_sample(10, 11, 0, None, None) == L.CSC_E_INVALID


@pytest.mark.parametrize("m", [0, 1, 5, 50, 100])
@pytest.mark.parametrize("lam", [0.0, 0.013, 0.4375, 1.0, 1.93, 2.0])
@pytest.mark.parametrize("flags", [0, 2])
def test_coefficients_match_oracle(L, m, lam, flags):
    c = np.empty(m + 1)
    assert L.lib().csc_chebyshev_coefficients(lam, m, flags, c.ctypes.data_as(ctypes.c_void_p)) == 0
    ref = och.filter_coeffs(lam, m, damped=(flags == 0))
    assert np.allclose(c, ref, rtol=1e-13, atol=1e-15)


def test_eigencount_matches_oracle(L):
    rng = np.random.default_rng(0)
    mu = rng.normal(size=51) * 10
    mu[0] = 1000.0
    for lam in (0.0, 0.3, 1.1, 2.0):
        out = ctypes.c_double()
        assert L.lib().csc_eigencount(mu.ctypes.data_as(ctypes.c_void_p), 50, lam, 0, ctypes.byref(out)) == 0
        assert out.value == pytest.approx(och.eigencount(mu, lam), rel=1e-12, abs=1e-9)


def test_workload_defaults_agree():
    import paper_1602_02018_gb300 as csc
    from oracle import pipeline

    for n_nodes, k in ((1000, 20), (100_000, 200), (10**6, 100)):
        a = csc.default_sizes(n_nodes, k)
        b = pipeline.defaults(n_nodes, k)
        w = ci.workload_sizes(n_nodes, k)
        assert a["d"] == b["d"] == w["d"] and a["n"] == b["n"] == w["n"] and a["n_probes"] == b["n_v"] == w["n_v"]


def test_sweep_tables_format():
    """The recovery-sweep report renders every table from a result dictionary."""
    from tests import fig1_sweep as fs

    var = fs.variants()
    row = dict(csc={("def", None): 0.9, ("hp", None): 0.95}, sc=1.0, lam_est=0.4, lk=0.3, lk1=0.5, est_in_gap=1.0)
    for f, (_, vals) in var.items():
        for v in vals:
            row["csc"][(f, v)] = 0.8
    res = {"hom": {0.02: row}, "het": {0.0: row},
           "fg": {(1000, 20): {t: dict(ari=0.9, ms=4.0, wall_s=0.004) for t in ("l4", "hp", "hp200")}},
           "fg_sc": dict(ari=0.99, sec=0.3)}
    text = fs.format_tables(res, 3)
    for needle in ("Fig. 1 a", "Fig. 1 d", "Fig. 1 e", "Heterogeneous SBM", "Fig. 1 f-g", "SC (Alg. 1"):
        assert needle in text


def test_sampling_wrappers_reject_bad_output_buffers():
    """The sampling wrappers check the caller's index buffer before any native call: it must be a
    contiguous int64 CUDA tensor of at least n elements (anything else would be written past)."""
    import pytest
    import torch

    import paper_1602_02018_gb300 as csc

    for fn in (csc.csc_sample, csc.csc_sample_noalloc):
        with pytest.raises(ValueError):
            fn(100, 10, 0, torch.empty(10, dtype=torch.int64))  # host memory
        with pytest.raises(ValueError):
            fn(100, 10, 0, torch.empty(10, dtype=torch.int32))
