"""k-means on the reduced feature set (Alg. 2 step 6), test infrastructure only.

The paper runs Matlab's kmeans with 20 replicates (Sec. 5) and the default
maximum of 100 iterations (Sec. 5.2), Euclidean distance.  Reading of the
parts the paper leaves to that library:

* seeding: k-means++ (Arthur & Vassilvitskii 2007).  Replicate r draws its
  uniforms from Philox (stream STREAM_KMEANS, counter (r, t)): the first
  centre is point floor(u n); centre t >= 1 is the first point whose
  cumulative squared distance to the chosen centres reaches u * total.
* Lloyd iterations: assign every point to its nearest centre (ties to the
  lowest centre index), move every centre to the mean of its points, stop
  when no assignment changes or after ``max_iter`` updates.
* an empty cluster, taken in increasing index, gets the point farthest from
  its own centre (ties to the lowest point index), which moves to it.
* the replicate with the smallest inertia sum ||x_i - c_label(i)||^2 wins
  (ties to the first).

Pins (tests/test_oracle_misc.py): on n <= 10 points with k <= 3 the best
replicate reaches the minimum inertia found by brute force over all
partitions; well-separated blobs are recovered exactly.
"""
from __future__ import annotations

import numpy as np

from .rng import STREAM_KMEANS, uniform_draw


def _sqdist(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    return np.sum((x[:, None, :] - c[None, :, :]) ** 2, axis=2)


def kmeanspp(x: np.ndarray, k: int, seed: int, rep: int) -> np.ndarray:
    n = x.shape[0]
    idx = [min(int(uniform_draw(seed, STREAM_KMEANS, rep, 0) * n), n - 1)]
    d2 = np.sum((x - x[idx[0]]) ** 2, axis=1)
    for t in range(1, k):
        u = uniform_draw(seed, STREAM_KMEANS, rep, t)
        total = float(np.sum(d2))
        if total <= 0.0:
            p = min(int(u * n), n - 1)
        else:
            cum = np.cumsum(d2)
            p = int(np.searchsorted(cum, u * total, side="left"))
            p = min(p, n - 1)
        idx.append(p)
        d2 = np.minimum(d2, np.sum((x - x[p]) ** 2, axis=1))
    return x[np.array(idx)].copy()


def lloyd(x: np.ndarray, centers: np.ndarray, max_iter: int):
    k = centers.shape[0]
    c = centers.copy()
    lab = np.argmin(_sqdist(x, c), axis=1)
    it = 0
    for it in range(1, max_iter + 1):
        newc = np.zeros_like(c)
        cnt = np.bincount(lab, minlength=k)
        np.add.at(newc, lab, x)
        nonempty = cnt > 0
        newc[nonempty] /= cnt[nonempty, None]
        for j in np.nonzero(~nonempty)[0]:
            dist = np.sum((x - newc[lab]) ** 2, axis=1)
            p = int(np.argmax(dist))
            newc[j] = x[p]
            lab[p] = j
        c = newc
        new_lab = np.argmin(_sqdist(x, c), axis=1)
        if np.array_equal(new_lab, lab):
            lab = new_lab
            break
        lab = new_lab
    inertia = float(np.sum((x - c[lab]) ** 2))
    return lab.astype(np.int32), c, inertia, it


def kmeans(x: np.ndarray, k: int, replicates: int = 20, max_iter: int = 100, seed: int = 0):
    """Best of ``replicates`` k-means runs: (labels int32[n], centers, inertia, iterations)."""
    x = np.asarray(x, dtype=np.float64)
    best = None
    for r in range(replicates):
        c0 = kmeanspp(x, k, seed, r)
        lab, c, inertia, it = lloyd(x, c0, max_iter)
        if best is None or inertia < best[2]:
            best = (lab, c, inertia, it)
    return best
