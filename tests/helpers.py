"""Shared helpers of the parity tests (inputs from csc_inputs, expectations from oracle/)."""
import numpy as np

import csc_inputs as ci


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def small_graphs():
    """Edge cases and ragged sizes: (name, CSRGraph)."""
    out = []
    out.append(("single_node", ci.from_edges(1, np.array([], np.int64), np.array([], np.int64))))
    out.append(("pair", ci.from_edges(2, np.array([0]), np.array([1]))))
    out.append(("path7", ci.path(7)))
    out.append(("ring33", ci.ring(33)))
    iso = ci.from_edges(9, np.array([0, 1, 2, 5]), np.array([1, 2, 3, 6]))  # isolated nodes 4, 7, 8
    out.append(("isolated", iso))
    out.append(("cliques", ci.disjoint_cliques(5, 7)))
    out.append(("sbm1000", ci.sbm(1000, 20, seed=0)))
    out.append(("er777", ci.erdos_renyi(777, 0.02, seed=3)))
    return out


def with_self_loops(g):
    """Copy of g's CSR with a self loop inserted in every third row (kept sorted)."""
    rp, cols = [0], []
    for i in range(g.n):
        row = list(g.col_idx[g.row_ptr[i]:g.row_ptr[i + 1]])
        if i % 3 == 0:
            row = sorted(row + [i])
        cols.extend(row)
        rp.append(len(cols))
    return np.array(rp, np.int64), np.array(cols, np.int32)
