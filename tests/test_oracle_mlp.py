"""Pins of the FP64 perceptron reference and of the line features (CPU only)."""
import numpy as np
import pytest

from oracle import evs, features, mlp
from paper_0807_1949_gb300 import inputs


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, mlp.NPARAMS)


def test_finite_differences():
    p = _params(0)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(7, 8))
    t = rng.normal(size=7)
    _, g = mlp.loss_and_grad(p, X, t)
    h = 1e-6
    for k in rng.choice(mlp.NPARAMS, size=60, replace=False):
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss_and_grad(p + e, X, t)[0] - mlp.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_all_active_regime_is_affine():
    """Positive weights and inputs keep every ReLU active: y = W3 (W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(2)
    d = {"W1": rng.uniform(0.1, 1, (64, 8)), "b1": rng.uniform(0.1, 1, 64), "W2": rng.uniform(0.1, 1, (64, 64)),
         "b2": rng.uniform(0.1, 1, 64), "W3": rng.normal(size=64), "b3": np.array([0.3])}
    p = mlp.pack(d)
    X = rng.uniform(0.1, 1, (5, 8))
    t = rng.normal(size=5)
    y, _ = mlp.forward(p, X)
    M = d["W3"] @ d["W2"] @ d["W1"]
    c = d["W3"] @ (d["W2"] @ d["b1"] + d["b2"]) + d["b3"][0]
    assert np.allclose(y, X @ M + c, rtol=1e-12)
    _, g = mlp.loss_and_grad(p, X, t)
    r = 2 * (y - t) / len(t)
    gd = mlp.unpack(g)
    assert np.isclose(gd["b3"][0], r.sum())
    assert np.allclose(gd["W1"], np.outer(d["W3"] @ d["W2"], r @ X), rtol=1e-10)


def test_bf16_rounding():
    """bfloat16 keeps 8 significant bits: near 1 the spacing is 2^-7; halfway cases go to even."""
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -9, 1 + 3 * 2 ** -9, -2.5, 3.1415927], np.float32)
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                  # tie between 1 and 1 + 2^-7 -> even mantissa
    assert r[2] == 1 + 2 ** -6          # tie between 1 + 2^-7 and 1 + 2^-6 -> even mantissa
    assert r[3] == 1.0 and r[4] == 1 + 2 ** -7
    assert r[5] == -2.5 and r[6] == 3.140625


def test_adam_first_step():
    rng = np.random.default_rng(3)
    p, g = rng.normal(size=10), rng.normal(size=10)
    p1, _, _ = mlp.adam_step(p, np.zeros(10), np.zeros(10), g, 1, lr=0.01, eps=1e-8)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_line_features_small_grid():
    dims = (9, 8)
    A = inputs.grid_poisson(dims, sigma=0.0)
    split = evs.split_grid(A, dims, (4, 4))
    f = features.line_features(split, A)
    assert f.shape == (2 * len(split.vtl), 8)
    # constant-coefficient Laplacian: a_ii = 4 everywhere, neighbours all 1
    assert np.allclose(f[:, 0], np.log(4.0))
    assert np.allclose(f[:, 6], 0.0)
    # the corner (4, 4) has 4 copies with 2 lines each
    corner_rows = [2 * t + s for t, q in enumerate(split.vtl) for s in (0, 1)
                   if split.subgraphs[q[2 * s]].vertices[q[2 * s + 1]] == 4 + 9 * 4]
    assert len(corner_rows) == 8
    assert np.allclose(f[corner_rows, 2], np.log(4)) and np.allclose(f[corner_rows, 3], 2)
