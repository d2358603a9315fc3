"""FP64 reference of the learned-impedance perceptron — TEST INFRASTRUCTURE ONLY.

The paper has no network: §7 makes the impedances the preconditioner and §7.1 gives a matching
rule; the project's model predicts log Z of a line end from 8 local features.  This module is the
plain FP64 definition the GPU kernels are checked against:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 . h2 + b3          (8 -> 64 -> 64 -> 1)
    loss = mean_i (y_i - t_i)^2

evaluated with the weights rounded to bfloat16 (round to nearest, ties to even, as the kernels
hold them), and the gradient of the loss with respect to those weights by the chain rule.
Adam follows Kingma & Ba (2015), Algorithm 1, with bias correction.

Parameter layout (4801 values): W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.

Pins: central finite differences of ``loss_and_grad``; the all-active regime where the network is
the affine map W3 (W2 (W1 x + b1) + b2) + b3 with its closed-form gradient; the first Adam step
moves every parameter by lr * g / (|g| + eps).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 64
SIZES = [("W1", NH * NIN), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("W3", NH), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, size in SIZES:
        out[name] = p[o:o + size]
        o += size
    out["W1"] = out["W1"].reshape(NH, NIN)
    out["W2"] = out["W2"].reshape(NH, NH)
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16_round(p) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even) and return them as float64."""
    a = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(p: np.ndarray, X: np.ndarray):
    """y (n,) and the cache for the backward pass; p already in the precision to use."""
    w = unpack(np.asarray(p, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w["W3"] + w["b3"][0]
    return y, (X, a1, h1, a2, h2, w)


def loss_and_grad(p: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient (chain rule), both FP64."""
    y, (X, a1, h1, a2, h2, w) = forward(p, X)
    n = len(y)
    err = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(err * err))
    dy = 2.0 * err / n
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    d2 = np.outer(dy, w["W3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def adam_step(p, m, v, g, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
