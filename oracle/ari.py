"""Adjusted Rand index (Hubert & Arabie 1985), the recovery score of Sec. 5.2.

Test infrastructure only.  ARI = (sum_ij C(n_ij, 2) - E) / (max_term - E) with
E = sum_i C(a_i, 2) sum_j C(b_j, 2) / C(n, 2) and max_term the mean of the two
marginal sums, over the contingency table n_ij of two labelings.

Pins (tests/test_oracle_misc.py): identical labelings give 1; relabelling
is invisible; hand-computed contingency tables.
"""
from __future__ import annotations

import numpy as np


def _c2(x):
    x = np.asarray(x, dtype=np.float64)
    return x * (x - 1) / 2.0


def ari(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        raise ValueError("label arrays differ in length")
    n = a.size
    if n < 2:
        return 1.0
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1))
    np.add.at(table, (ai, bi), 1)
    sum_ij = _c2(table).sum()
    sa = _c2(table.sum(axis=1)).sum()
    sb = _c2(table.sum(axis=0)).sum()
    expected = sa * sb / _c2(n)
    max_term = 0.5 * (sa + sb)
    if max_term == expected:
        return 1.0
    return float((sum_ij - expected) / (max_term - expected))
