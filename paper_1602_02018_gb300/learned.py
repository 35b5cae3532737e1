"""Learned lambda_k bracket: training data, training and use.

Every step runs in libcsc: the features and the eigencount moments
(csc_bracket_features, csc_kpm_moments), the target crossings
(csc_bracket_target), the fit -- targets, standardisation constants, training
and the calibration of the half-width factor (csc_bracket_fit) -- the
predictions (csc_bracket_predict) and the bracketed dichotomy
(csc_estimate_lambda_k_learned).  This module only gathers the arrays and
keeps the fitted constants together.

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

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from . import api as csc

_RULES = {"evaluations": 0, "coverage": 1}


def bracket_sample(g: csc.Graph, k: int, m: int = 50, n_probes: int = 0, seed: int = 0):
    """(features float32[72], target bracket (lo, hi)) of one graph handle; n_probes 0 ->
    the library's default ceil(2 ln N)."""
    feat, _ = csc.csc_bracket_features(g, k, seed)
    mu = csc.csc_kpm_moments(g, m + 1, n_probes, seed)
    lo, hi = csc.csc_bracket_target(mu, k)
    return feat, (lo, hi)


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
        """Train on all but the last ``val_frac`` of the samples (csc_bracket_fit); ``widen``
        is calibrated on those held-back samples: by default to the fewest mean
        eigencount evaluations of the started halving, or with ``widen_rule="coverage"``
        so that a ``coverage`` share of their brackets is met."""
        params, norm, widen, n_fit, hist = csc.csc_bracket_fit(feats, brackets, val_frac, epochs, batch, lr, seed,
                                                               _RULES[widen_rule], coverage)
        return cls(params, norm, widen, hist, n_fit, len(feats) - n_fit)

    def predict_targets(self, feats: np.ndarray) -> np.ndarray:
        """(centre, ln half-width) per row of raw features."""
        return csc.csc_bracket_predict(self.params, self.norm, self.widen, feats)[0]

    def predict_brackets(self, feats: np.ndarray) -> np.ndarray:
        """The brackets csc_estimate_lambda_k_learned starts from, per row of raw features."""
        return csc.csc_bracket_predict(self.params, self.norm, self.widen, feats)[1]

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


def dataset(graphs: Sequence, m: int = 50, seed: int = 0, flags: int = 0):
    """Features and target brackets of (CSRGraph-like, k) pairs: (feats [n x 72], brackets [n x 2])."""
    feats, brs = [], []
    for g, k in graphs:
        with csc.csc_graph_create(g.row_ptr, g.col_idx, flags) as h:
            f, b = bracket_sample(h, k, m, 0, seed)
        feats.append(f)
        brs.append(b)
    return np.stack(feats), np.array(brs, dtype=np.float64)
