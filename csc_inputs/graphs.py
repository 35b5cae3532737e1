"""Seeded random graphs in CSR form.

Every generator returns an undirected, unweighted simple graph (no self
loops, no duplicate edges) as a symmetric CSR with sorted column indices:
``row_ptr`` int64[N+1], ``col_idx`` int32[nnz] with nnz = 2 * #edges.

* ``sbm``: stochastic block model of Sec. 5.1 -- edge probability q1 inside a
  community and q2 = eps * q1 across communities, parameterised by the ratio
  eps and the mean degree s.  Edges are drawn exactly: for each block (and
  once for all cross-block pairs) the edge count is Binomial(#pairs, q) and a
  uniformly random subset of pairs of that size is taken.
* ``chung_lu``: expected-degree (Chung-Lu) graph with p_ij = min(1, w_i w_j / sum(w)),
  drawn exactly by the Miller-Hagberg skipping scheme (Miller & Hagberg 2011),
  vectorised over source nodes.
* small textbook graphs (ring, complete, cliques, path, bipartite) used as
  spectral pins.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np


@dataclass
class CSRGraph:
    row_ptr: np.ndarray  # int64 [N+1]
    col_idx: np.ndarray  # int32 [nnz]
    labels: Optional[np.ndarray] = None  # int32 [N] ground-truth community, if any
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def edges(self):
        """Upper-triangle edge list (i < j)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        cols = self.col_idx.astype(np.int64)
        keep = rows < cols
        return rows[keep], cols[keep]


def from_edges(n: int, i: np.ndarray, j: np.ndarray, labels=None, meta=None) -> CSRGraph:
    """Symmetric CSR from an undirected edge list; drops self loops and duplicates."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    keep = i != j
    i, j = i[keep], j[keep]
    a = np.minimum(i, j)
    b = np.maximum(i, j)
    if a.size:
        key = np.unique(a * n + b)
        a, b = key // n, key % n
    rows = np.concatenate([a, b])
    cols = np.concatenate([b, a])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    lab = None if labels is None else np.asarray(labels, dtype=np.int32)
    return CSRGraph(row_ptr, cols.astype(np.int32), lab, dict(meta or {}))


# ---------------------------------------------------------------------------
# Stochastic block model (Sec. 5.1)
# ---------------------------------------------------------------------------

def epsilon_c(s: float, k: int) -> float:
    """Critical ratio eps_c = (s - sqrt(s)) / (s + sqrt(s)(k - 1)) (Sec. 5.1, Decelle et al.)."""
    r = np.sqrt(s)
    return (s - r) / (s + r * (k - 1))


def sbm_probabilities(sizes: Sequence[int], s: float, eps: float):
    """(q1, q2) such that the expected mean degree is s and q2 = eps * q1."""
    sizes = np.asarray(sizes, dtype=np.float64)
    n = sizes.sum()
    denom = np.sum(sizes * ((sizes - 1.0) + eps * (n - sizes))) / n
    q1 = s / denom
    return q1, eps * q1


def _tri_decode(t: np.ndarray, m: int):
    """Map pair index t in [0, m(m-1)/2) to (a, b), 0 <= a < b < m, row-major over a."""
    t = t.astype(np.int64)
    # a = largest a with a*m - a(a+1)/2 <= t
    mf = float(m)
    a = np.floor((2 * mf - 1 - np.sqrt((2 * mf - 1) ** 2 - 8.0 * t)) / 2).astype(np.int64)
    a = np.clip(a, 0, m - 2)
    start = a * m - a * (a + 1) // 2
    # fix rounding at boundaries
    over = start > t
    while np.any(over):
        a[over] -= 1
        start = a * m - a * (a + 1) // 2
        over = start > t
    nxt = (a + 1) * m - (a + 1) * (a + 2) // 2
    under = nxt <= t
    while np.any(under):
        a[under] += 1
        start = a * m - a * (a + 1) // 2
        nxt = (a + 1) * m - (a + 1) * (a + 2) // 2
        under = nxt <= t
    b = a + 1 + (t - start)
    return a, b


def sbm(n: int, k: int, s: float = 16.0, eps: Optional[float] = None, seed: int = 0,
        sizes: Optional[Sequence[int]] = None, eps_over_epsc: float = 0.25) -> CSRGraph:
    """Stochastic block model with k communities and mean degree s.

    Communities are contiguous node ranges (node order = generation order).
    ``eps`` defaults to eps_c/4, the setting of the paper's Fig. 1 f-g.
    ``sizes`` gives heterogeneous community sizes (supplementary experiment).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if sizes is None:
        if n % k:
            raise ValueError("n must be a multiple of k for equal communities")
        sizes = [n // k] * k
    sizes = np.asarray(sizes, dtype=np.int64)
    if int(sizes.sum()) != n:
        raise ValueError("community sizes must sum to n")
    if eps is None:
        eps = eps_over_epsc * epsilon_c(s, k)
    q1, q2 = sbm_probabilities(sizes, s, eps)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    labels = np.repeat(np.arange(k, dtype=np.int32), sizes)
    ei, ej = [], []
    # intra-community edges, exact: Binomial count then a uniform subset of pairs
    for b in range(k):
        m = int(sizes[b])
        pairs = m * (m - 1) // 2
        if pairs == 0:
            continue
        c = int(rng.binomial(pairs, min(q1, 1.0)))
        if c == 0:
            continue
        t = rng.choice(pairs, size=c, replace=False)
        a, bb = _tri_decode(t, m)
        ei.append(a + starts[b])
        ej.append(bb + starts[b])
    # inter-community edges, exact: Binomial count then uniform distinct cross pairs
    total_pairs = (n * (n - 1)) // 2 - int(np.sum(sizes * (sizes - 1) // 2))
    if total_pairs > 0 and q2 > 0:
        c = int(rng.binomial(total_pairs, min(q2, 1.0)))
        got = np.empty(0, dtype=np.int64)
        while got.size < c:
            need = c - got.size
            draw = int(need * 1.3) + 64
            i = rng.integers(0, n, size=draw)
            j = rng.integers(0, n, size=draw)
            keep = labels[i] != labels[j]
            i, j = i[keep], j[keep]
            key = np.minimum(i, j) * n + np.maximum(i, j)
            key = np.unique(np.concatenate([got, key]))
            got = key
        if got.size > c:
            got = rng.choice(got, size=c, replace=False)
        ei.append(got // n)
        ej.append(got % n)
    i = np.concatenate(ei) if ei else np.empty(0, np.int64)
    j = np.concatenate(ej) if ej else np.empty(0, np.int64)
    return from_edges(n, i, j, labels,
                      dict(kind="sbm", n=n, k=k, s=s, eps=float(eps), q1=float(q1),
                           q2=float(q2), seed=seed))


# ---------------------------------------------------------------------------
# Chung-Lu power-law graph
# ---------------------------------------------------------------------------

def _pareto_mean(alpha: float, w_max: float) -> float:
    """Mean of a Pareto(1, alpha) law truncated to [1, w_max]."""
    if abs(alpha - 1.0) < 1e-9:
        return np.log(w_max) / (1.0 - 1.0 / w_max)
    return alpha * (1 - w_max ** (1 - alpha)) / ((alpha - 1) * (1 - w_max ** (-alpha)))


def chung_lu_weights(n: int, exponent: float = 2.1, mean: float = 6.0, w_min: float = 1.0,
                     cutoff: Optional[float] = None):
    """Deterministic quantiles of a truncated Pareto law with mean ``mean``.

    Degree exponent gamma gives tail index alpha = gamma - 1.  Without
    ``cutoff`` the lower end is ``w_min`` and the truncation point w_max solves
    E[w] = mean by bisection.  With ``cutoff`` the upper end is w_max = cutoff
    and the lower end w_min solves E[w] = mean instead (for exponents whose
    untruncated mean with w_min = 1 is below ``mean``).  Node i gets the
    quantile at u = (i + 0.5) / n, so weights are sorted ascending.
    """
    alpha = exponent - 1.0
    if cutoff is None:
        lo, hi = 1.0 + 1e-9, 1e12
        if _pareto_mean(alpha, hi) * w_min < mean:
            raise ValueError("mean degree unreachable for this exponent")
        for _ in range(200):
            mid = np.sqrt(lo * hi)
            if _pareto_mean(alpha, mid) * w_min < mean:
                lo = mid
            else:
                hi = mid
        ratio = hi
    else:
        if not cutoff > mean:
            raise ValueError("cutoff must exceed the mean")
        # E[w] = w_min * mean(ratio = cutoff / w_min) is increasing in w_min
        lo, hi = 1e-12, float(mean)
        for _ in range(200):
            mid = np.sqrt(lo * hi)
            if mid * _pareto_mean(alpha, cutoff / mid) < mean:
                lo = mid
            else:
                hi = mid
        w_min = hi
        ratio = cutoff / w_min
    u = (np.arange(n, dtype=np.float64) + 0.5) / n
    w = w_min * (1.0 - u * (1.0 - ratio ** (-alpha))) ** (-1.0 / alpha)
    return w, ratio * w_min


def _components(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Connected-component label of every node (union-find over the edge list)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg

    a = sp.coo_matrix((np.ones(src.size), (src, dst)), shape=(n, n))
    return csg.connected_components(a, directed=False)[1]


def chung_lu(n: int, exponent: float = 2.1, mean: float = 6.0, seed: int = 0,
             min_degree_one: bool = True, connect: bool = True, cutoff: Optional[float] = None) -> CSRGraph:
    """Chung-Lu graph with p_ij = min(1, w_i w_j / sum(w)), drawn exactly.

    Miller-Hagberg: with weights sorted descending, each source u walks the
    candidates v > u with geometric skips under the current bound p and
    accepts with probability q/p.  All sources advance together, so the cost
    is O(n + #edges) numpy work.  With ``min_degree_one`` every node left
    isolated gets one edge to a node drawn with probability proportional to
    its weight, so the minimum degree is 1.  With ``connect`` every connected
    component other than the largest gets one more edge, from a node drawn
    uniformly in it to a node of the largest component drawn with probability
    proportional to its weight, so the graph is connected.  ``cutoff`` fixes
    the largest weight instead of the smallest (see ``chung_lu_weights``).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w_asc, w_max = chung_lu_weights(n, exponent, mean, cutoff=cutoff)
    order = np.argsort(-w_asc, kind="stable")  # descending
    w = w_asc[order]
    total = w.sum()
    src_all, dst_all = [], []
    u = np.arange(n - 1, dtype=np.int64)
    v = u + 1
    p = np.minimum(w[u] * w[v] / total, 1.0)
    active = np.ones(u.size, dtype=bool)
    while True:
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        uu, vv, pp = u[idx], v[idx], p[idx]
        r = rng.random(idx.size)
        with np.errstate(divide="ignore", invalid="ignore"):
            skip = np.where(pp >= 1.0, 0.0, np.floor(np.log(r) / np.log1p(-pp)))
        skip = np.where(pp <= 0.0, float(n), skip)
        vv = vv + np.minimum(skip, float(n)).astype(np.int64)
        alive = vv < n
        vv_c = np.minimum(vv, n - 1)
        q = np.minimum(w[uu] * w[vv_c] / total, 1.0)
        r2 = rng.random(idx.size)
        acc = alive & (r2 < q / np.maximum(pp, 1e-300))
        src_all.append(uu[acc])
        dst_all.append(vv[acc])
        v[idx] = vv + 1
        p[idx] = q
        still = alive & (vv + 1 < n)
        active[idx] = still
    src = np.concatenate(src_all) if src_all else np.empty(0, np.int64)
    dst = np.concatenate(dst_all) if dst_all else np.empty(0, np.int64)
    # back to ascending-weight node ids
    src = order[src]
    dst = order[dst]
    if min_degree_one:
        deg = np.bincount(np.concatenate([src, dst]), minlength=n)
        iso = np.nonzero(deg == 0)[0]
        if iso.size:
            cdf = np.cumsum(w_asc) / total
            tgt = np.searchsorted(cdf, rng.random(iso.size), side="right")
            tgt = np.minimum(tgt, n - 1)
            same = tgt == iso
            tgt[same] = (tgt[same] + 1) % n
            src = np.concatenate([src, iso])
            dst = np.concatenate([dst, tgt])
    if connect and n > 1:
        comp = _components(n, src, dst)
        sizes = np.bincount(comp)
        giant = int(np.argmax(sizes))
        others = np.nonzero(np.arange(sizes.size) != giant)[0]
        if others.size:
            # one node per small component, uniformly within it
            order = np.argsort(comp, kind="stable")
            starts = np.concatenate([[0], np.cumsum(sizes)])
            pick = starts[others] + (rng.random(others.size) * sizes[others]).astype(np.int64)
            a_nodes = order[pick]
            gnodes = np.nonzero(comp == giant)[0]
            cdf = np.cumsum(w_asc[gnodes]) / np.sum(w_asc[gnodes])
            b_nodes = gnodes[np.minimum(np.searchsorted(cdf, rng.random(others.size), side="right"),
                                        gnodes.size - 1)]
            src = np.concatenate([src, a_nodes])
            dst = np.concatenate([dst, b_nodes])
    return from_edges(n, src, dst, None,
                      dict(kind="chung_lu", n=n, exponent=exponent, mean=mean,
                           w_max=float(w_max), seed=seed))


# ---------------------------------------------------------------------------
# Small textbook graphs (spectral pins)
# ---------------------------------------------------------------------------

def ring(n: int) -> CSRGraph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, meta=dict(kind="ring"))


def path(n: int) -> CSRGraph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, meta=dict(kind="path"))


def complete(n: int) -> CSRGraph:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, meta=dict(kind="complete"))


def complete_bipartite(a: int, b: int) -> CSRGraph:
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return from_edges(a + b, i.ravel(), j.ravel(), meta=dict(kind="bipartite"))


def disjoint_cliques(k: int, size: int) -> CSRGraph:
    ei, ej = [], []
    for b in range(k):
        i, j = np.triu_indices(size, 1)
        ei.append(i + b * size)
        ej.append(j + b * size)
    labels = np.repeat(np.arange(k), size)
    return from_edges(k * size, np.concatenate(ei), np.concatenate(ej), labels,
                      dict(kind="cliques", k=k, size=size))


def erdos_renyi(n: int, p: float, seed: int = 0) -> CSRGraph:
    rng = np.random.Generator(np.random.PCG64(seed))
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.size) < p
    return from_edges(n, i[keep], j[keep], meta=dict(kind="er", p=p, seed=seed))


def block_diagonal(graphs: Sequence[CSRGraph]) -> CSRGraph:
    """Concatenate graphs into one block-diagonal CSR (node ids shifted)."""
    offs = np.concatenate([[0], np.cumsum([g.n for g in graphs])]).astype(np.int64)
    rps, cis, labs = [np.zeros(1, np.int64)], [], []
    base = 0
    lab_base = 0
    for g, o in zip(graphs, offs[:-1]):
        rps.append(g.row_ptr[1:] + base)
        cis.append(g.col_idx.astype(np.int64) + o)
        base += g.nnz
        if g.labels is not None:
            labs.append(g.labels.astype(np.int64) + lab_base)
            lab_base += int(g.labels.max()) + 1 if g.labels.size else 0
    labels = np.concatenate(labs).astype(np.int32) if len(labs) == len(graphs) else None
    return CSRGraph(np.concatenate(rps), np.concatenate(cis).astype(np.int32), labels,
                    dict(kind="block_diagonal", offsets=offs))
