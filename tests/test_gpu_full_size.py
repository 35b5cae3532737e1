"""The filter at the power-law workload's full size (Chung-Lu N = 1e6, degree exponent
2.1, mean degree 6, RCM-reordered CSR, m = 100, d = 56, Clenshaw form, autotuned launch
shape as bench.py runs it), checked on sampled outputs: the columns of Y = h~(L) R are
independent, so the FP64 oracle filters two sampled columns alone (Sec. 2.1 recurrence)
and they are compared with the GPU's whole-block result."""
import numpy as np
import pytest
import torch

import csc_inputs as ci
from oracle import chebyshev as och
from oracle import laplacian as olap

from .helpers import rel

pytestmark = pytest.mark.gpu

csc = pytest.importorskip("paper_1602_02018_gb300")

N, D, M, LAM = 1_000_000, 56, 100, 0.0597
COLS = [0, 37]


@pytest.fixture(scope="module")
def c3():
    from paper_1602_02018_gb300 import build

    build.build()
    g = ci.chung_lu(N, exponent=2.1, mean=6.0, seed=0)
    r = ci.gaussian_block(N, D, D, seed=21)
    s = olap.normalized_adjacency(g.row_ptr, g.col_idx)
    ref = och.cheb_filter(s, r[:, COLS].astype(np.float64), och.filter_coeffs(LAM, M))
    return g, r, ref


@pytest.mark.parametrize("storage,tol", [(0, 1e-4), (1, 0.15)])  # F32, BF16 (signal block stored in bf16)
def test_chung_lu_1e6_sampled_columns(c3, storage, tol):
    g, r, ref = c3
    with csc.csc_graph_create(g.row_ptr, g.col_idx, csc.RCM) as h:
        y = csc.csc_filter_random_signals(h, LAM, M, D, D, storage=storage, R_in=torch.from_numpy(r).cuda(),
                                          flags=csc.CLENSHAW)
        yc = y[:, COLS].double().cpu().numpy()
    for i in range(len(COLS)):
        err = rel(yc[:, i], ref[:, i])
        assert err <= tol, f"column {COLS[i]}: relative error {err:.3g}"
