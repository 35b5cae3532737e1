"""Pins of the storage-rounding model (tests/storage_emulation.py) used to derive the
full-size tolerances: its bf16 rounding against torch's conversion, and its filter against
the FP64 oracle (Sec. 2.1 recurrence) -- close for FP32 storage, and the error growing as
the storage narrows."""
import numpy as np
import torch

import csc_inputs as ci
from oracle import chebyshev as och
from oracle import laplacian as olap

from .helpers import rel
from .storage_emulation import clenshaw_stored, round_bf16


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 20000),
                        # exact ties between two bf16 neighbours, both parities
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0],
                                 dtype=np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(round_bf16(x), ref)


def test_storage_model_against_oracle():
    g = ci.sbm(1000, 20, seed=0)
    r = ci.gaussian_block(g.n, 8, 8, seed=1).astype(np.float64)
    c = och.filter_coeffs(0.45, 50)
    ref = och.cheb_filter(olap.normalized_adjacency(g.row_ptr, g.col_idx), r, c)
    e32 = rel(clenshaw_stored(g.row_ptr, g.col_idx, r, c, "f32"), ref)
    e16 = rel(clenshaw_stored(g.row_ptr, g.col_idx, r, c, "bf16"), ref)
    assert 0 < e32 < 1e-5          # fp32 rounding only
    assert 1e-4 < e16 < 5e-2       # bf16 storage: about 2^-9 per stored value, accumulated
    # an isolated node keeps s = 1 and an empty neighbour sum, so (L - I) is 0 on it:
    # Y_i = sum_j c_j T_j(0) R_i = h~(1) R_i
    iso = ci.from_edges(3, np.array([0]), np.array([1]))
    ri = np.array([[1.0], [2.0], [3.0]])
    ci_ = och.filter_coeffs(0.7, 6)
    y = clenshaw_stored(iso.row_ptr, iso.col_idx, ri, ci_, "f32")
    assert abs(y[2, 0] - 3.0 * float(och.h_tilde(1.0, 0.7, 6))) < 1e-6
    assert rel(y, och.cheb_filter(olap.normalized_adjacency(iso.row_ptr, iso.col_idx), ri, ci_)) < 1e-6
