"""The bracket regressor: a 72 -> 256 -> 256 -> 2 ReLU perceptron (test infrastructure only).

The paper has no learned component; this is the reading used for the learned
lambda_k bracket.  Written out in FP64 with numpy matrix products:

* Parameters, one flat vector in this order: W1 [72 x 256] (row = input,
  column = output, row-major), b1 [256], W2 [256 x 256], b2 [256], W3 [256 x 2],
  b3 [2] -- 84,994 values.
* Forward: H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), Y = H2 W3 + b3
  (X is B x 72, one row per graph).
* Loss: smooth L1 with beta = 1 averaged over the B x 2 outputs:
  l(e) = e^2 / 2 if |e| < 1 else |e| - 1/2, e = Y - T.
* Backward: dY = clip(e, -1, 1) / (2B); dW3 = H2^T dY, db3 = column sums of dY;
  dH2 = dY W3^T masked by H2 > 0; the same two rules for layers 2 and 1
  (the derivative of relu at 0 is taken as 0).
* Adam (Kingma & Ba 2015): beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias
  corrected: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pins (tests/test_oracle_mlp.py): the gradient against central finite
differences of the loss (an independent route to the same derivative);
smooth-L1 values at hand-computed points; the first Adam step equals
-lr g / (|g| + eps) per coordinate; a network set by hand to compute a known
function.
"""
from __future__ import annotations

import numpy as np

SIZES = (72, 256, 256, 2)


def layout():
    """(name, shape) of each parameter block, in storage order."""
    out = []
    for i in range(3):
        out.append((f"W{i + 1}", (SIZES[i], SIZES[i + 1])))
        out.append((f"b{i + 1}", (SIZES[i + 1],)))
    return out


N_PARAMS = sum(int(np.prod(s)) for _, s in layout())


def unpack(params: np.ndarray) -> dict:
    p = np.asarray(params, dtype=np.float64)
    out, off = {}, 0
    for name, shape in layout():
        size = int(np.prod(shape))
        out[name] = p[off:off + size].reshape(shape)
        off += size
    return out


def pack(blocks: dict) -> np.ndarray:
    return np.concatenate([np.asarray(blocks[name], dtype=np.float64).ravel() for name, _ in layout()])


def forward(params: np.ndarray, x: np.ndarray):
    """Returns (Y, cache) with cache = (X, H1, H2)."""
    w = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ w["W1"] + w["b1"], 0.0)
    h2 = np.maximum(h1 @ w["W2"] + w["b2"], 0.0)
    y = h2 @ w["W3"] + w["b3"]
    return y, (x, h1, h2)


def smooth_l1(y: np.ndarray, t: np.ndarray) -> float:
    e = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    a = np.abs(e)
    return float(np.mean(np.where(a < 1.0, 0.5 * e * e, a - 0.5)))


def loss_and_grad(params: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(loss, gradient as a flat vector in the parameter layout)."""
    w = unpack(params)
    y, (x, h1, h2) = forward(params, x)
    b = y.shape[0]
    loss = smooth_l1(y, t)
    dy = np.clip(y - t, -1.0, 1.0) / (2.0 * b)
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = (dy @ w["W3"].T) * (h2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"].T) * (h1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def adam_step(params: np.ndarray, grad: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t >= 1; returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
