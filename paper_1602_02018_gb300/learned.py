"""Learned lambda_k bracket: training data, training and use.

Every step on a graph runs in libcsc: the features and the eigencount moments
(csc_bracket_features, csc_kpm_moments), the target crossings
(csc_bracket_target), the network's training and inference (csc_mlp_*), and
the bracketed dichotomy (csc_estimate_lambda_k_learned, which also applies the
input standardisation and the output transform at inference).  What this module
computes on the host is pre- and post-processing of the training set of this
add-on, which the paper does not have: the mean and standard deviation of the
training features and targets (the constants handed to the library), the
conversion of target brackets to (centre, ln half-width), the standardised
training arrays, and the calibration of the half-width factor ``widen`` by a
search over held-back samples.

Readings (the paper has no learned component): the regression target of a
graph is (centre, ln half-width) of the interval where its eigencount, from
degree-m moments of the full probe count, lies in [k - 1/2, k + 1/2]; features
and targets are standardised by their training mean and standard deviation (a
feature of zero spread maps to 0); the predicted half-width is multiplied by
a factor ``widen`` calibrated on samples held back from the fit, to the value
with the fewest eigencount evaluations of the halving started from the
prediction (or to reach a chosen share of their brackets).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import api as csc
from ._native import CSC_MLP_IN, CSC_MLP_OUT


def default_probes(n: int) -> int:
    return max(1, math.ceil(2 * math.log(n))) if n > 1 else 1


def bracket_sample(g: csc.Graph, k: int, m: int = 50, n_probes: int = 0, seed: int = 0):
    """(features float32[72], target bracket (lo, hi)) of one graph handle."""
    feat, _ = csc.csc_bracket_features(g, k, seed)
    nv = n_probes or default_probes(g.N)
    mu = csc.csc_kpm_moments(g, m + 1, nv, seed)
    lo, hi = csc.csc_bracket_target(mu, k)
    return feat, (lo, hi)


def bracket_targets(brackets: np.ndarray) -> np.ndarray:
    """[lo, hi] rows -> (centre, ln half-width) rows."""
    b = np.asarray(brackets, dtype=np.float64)
    return np.stack([0.5 * (b[:, 0] + b[:, 1]), np.log(np.maximum(0.5 * (b[:, 1] - b[:, 0]), 1e-12))], axis=1)


def _standardise(x: np.ndarray, mean: np.ndarray, std: np.ndarray) -> np.ndarray:
    safe = np.where(std > 0, std, 1.0)
    return np.where(std > 0, (x - mean) / safe, 0.0)


def needed_widen(pred_t: np.ndarray, brackets: np.ndarray) -> np.ndarray:
    """Per sample, the smallest half-width factor at which the predicted interval
    meets the target interval (0 when the predicted centre lies inside it)."""
    c, hw = pred_t[:, 0], np.exp(pred_t[:, 1])
    lo, hi = brackets[:, 0], brackets[:, 1]
    dist = np.where(c < lo, lo - c, np.where(c > hi, c - hi, 0.0))
    return dist / hw


def search_evaluations(c: float, hw: float, lo: float, hi: float) -> int:
    """Eigencount evaluations the halving started from the prediction (centre c,
    half-width hw) spends when the accepted cut-offs are exactly [lo, hi]: count
    rounds to k inside, exceeds k above, falls short below (a monotone count)."""
    def side(x):  # 0: accepted, +1: count above k, -1: below
        return 0 if lo <= x <= hi else (1 if x > hi else -1)

    def halve(a, b, n):
        for it in range(1, 61):
            mid = 0.5 * (a + b)
            sd = side(mid)
            if sd == 0:
                return n + it
            if sd > 0:
                b = mid
            else:
                a = mid
            if b - a < 1e-12 or it == 60:
                return n + it + 1
        return n + 60

    c = min(2.0, max(0.0, c))
    sc = side(c)
    if sc == 0:
        return 1
    e = max(0.0, c - hw) if sc > 0 else min(2.0, c + hw)
    se = side(e)
    if se == 0:
        return 2
    if sc > 0:
        return halve(e, c, 2) if se < 0 else halve(0.0, e, 2)
    return halve(c, e, 2) if se > 0 else halve(e, 2.0, 2)


def best_widen(pred_t: np.ndarray, brackets: np.ndarray, grid=None) -> float:
    """The half-width factor with the fewest mean evaluations of the started halving."""
    grid = np.geomspace(0.25, 4096.0, 57) if grid is None else grid
    hw = np.exp(np.minimum(pred_t[:, 1], 10.0))
    cost = [np.mean([search_evaluations(pred_t[i, 0], w * hw[i], brackets[i, 0], brackets[i, 1])
                     for i in range(len(hw))]) for w in grid]
    return float(grid[int(np.argmin(cost))])


@dataclass
class BracketModel:
    params: torch.Tensor  # device float32[CSC_MLP_PARAMS]
    norm: np.ndarray      # float32[148]: feature mean, feature std, target mean, target std
    widen: float = 1.0
    loss_history: Optional[np.ndarray] = None
    n_fit: int = 0
    n_val: int = 0

    @classmethod
    def fit(cls, feats: np.ndarray, brackets: np.ndarray, epochs: int = 300, batch: int = 32, lr: float = 1e-3,
            seed: int = 0, coverage: float = 0.9, val_frac: float = 0.15,
            widen_rule: str = "evaluations") -> "BracketModel":
        """Train on all but the last ``val_frac`` of the samples.  ``widen`` is calibrated
        on those held-back samples: by default to the fewest mean eigencount
        evaluations of the started halving (``search_evaluations``), or with
        ``widen_rule="coverage"`` so that a ``coverage`` share of their brackets is met."""
        feats = np.asarray(feats, dtype=np.float64)
        brackets = np.asarray(brackets, dtype=np.float64)
        n_val = int(round(val_frac * len(feats))) if len(feats) >= 10 else 0
        n_fit = len(feats) - n_val
        t = bracket_targets(brackets)
        fm, fs = feats[:n_fit].mean(axis=0), feats[:n_fit].std(axis=0)
        tm, ts = t[:n_fit].mean(axis=0), t[:n_fit].std(axis=0)
        ts = np.where(ts > 0, ts, 1.0)
        norm = np.concatenate([fm, fs, tm, ts]).astype(np.float32)
        # standardise with the float32 constants the library will use at inference
        fm32, fs32 = norm[:CSC_MLP_IN].astype(np.float64), norm[CSC_MLP_IN:2 * CSC_MLP_IN].astype(np.float64)
        x = _standardise(feats[:n_fit].astype(np.float32).astype(np.float64), fm32, fs32)
        x = torch.from_numpy(x.astype(np.float32)).cuda().contiguous()
        y = torch.from_numpy(((t[:n_fit] - tm) / ts).astype(np.float32)).cuda().contiguous()
        params = csc.csc_mlp_init(seed)
        hist = csc.csc_mlp_train(params, x, y, epochs, batch, lr, seed)
        model = cls(params, norm, 1.0, hist)
        cal = slice(n_fit, None) if n_val else slice(0, n_fit)
        pred = model.predict_targets(feats[cal])
        if widen_rule == "coverage":
            model.widen = float(max(1.0, np.quantile(needed_widen(pred, brackets[cal]), coverage)))
        else:
            model.widen = best_widen(pred, brackets[cal])
        model.n_fit, model.n_val = n_fit, n_val
        return model

    def predict_targets(self, feats: np.ndarray) -> np.ndarray:
        """(centre, ln half-width) per row of raw features (network run by libcsc)."""
        f = np.asarray(feats, dtype=np.float32).astype(np.float64)
        fm, fs = self.norm[:CSC_MLP_IN].astype(np.float64), self.norm[CSC_MLP_IN:2 * CSC_MLP_IN].astype(np.float64)
        x = torch.from_numpy(_standardise(f, fm, fs).astype(np.float32)).cuda().contiguous()
        y = csc.csc_mlp_forward(self.params, x).cpu().numpy().astype(np.float64)
        tm = self.norm[2 * CSC_MLP_IN:2 * CSC_MLP_IN + CSC_MLP_OUT].astype(np.float64)
        ts = self.norm[2 * CSC_MLP_IN + CSC_MLP_OUT:].astype(np.float64)
        return y * ts + tm

    def predict_brackets(self, feats: np.ndarray) -> np.ndarray:
        t = self.predict_targets(feats)
        hw = self.widen * np.exp(np.minimum(t[:, 1], 10.0))
        return np.stack([np.maximum(0.0, t[:, 0] - hw), np.minimum(2.0, t[:, 0] + hw)], axis=1)

    def estimate(self, g: csc.Graph, k: int, m: int = 50, n_probes: int = 0, seed: int = 0,
                 refilter: bool = False):
        return csc.csc_estimate_lambda_k_learned(g, k, self.params, self.norm, m, n_probes, seed, self.widen,
                                                 refilter)

    def save(self, path: str) -> None:
        np.savez(path, params=self.params.cpu().numpy(), norm=self.norm, widen=self.widen)

    @classmethod
    def load(cls, path: str) -> "BracketModel":
        z = np.load(path)
        return cls(torch.from_numpy(z["params"]).cuda(), z["norm"].astype(np.float32), float(z["widen"]))


def covered(pred: np.ndarray, brackets: np.ndarray) -> np.ndarray:
    """Whether each predicted interval meets its target interval."""
    return (pred[:, 0] <= brackets[:, 1]) & (pred[:, 1] >= brackets[:, 0])


def dataset(graphs: Sequence, m: int = 50, seed: int = 0, flags: int = 0):
    """Features and target brackets of (CSRGraph-like, k) pairs: (feats [n x 72], brackets [n x 2])."""
    feats, brs = [], []
    for g, k in graphs:
        with csc.csc_graph_create(g.row_ptr, g.col_idx, flags) as h:
            f, b = bracket_sample(h, k, m, 0, seed)
        feats.append(f)
        brs.append(b)
    return np.stack(feats), np.array(brs, dtype=np.float64)
