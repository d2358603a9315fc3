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


def _hand_grid():
    """A 5 x 5 five-point operator with chosen weights around two boundary vertices (ids x + 5 y):
    the edge copy 7 = (2, 1) on the cut line x = 2 and the corner 12 = (2, 2).  Every other edge has
    weight 1 and every other vertex the excess 0.5; a_ii = sum_j |a_ij| + delta_i."""
    import scipy.sparse as sp
    n = 25
    w = {}
    for y in range(5):
        for x in range(5):
            i = x + 5 * y
            if x < 4:
                w[(i, i + 1)] = 1.0
            if y < 4:
                w[(i, i + 5)] = 1.0
    w[(6, 7)], w[(7, 8)], w[(2, 7)], w[(7, 12)] = 1.0, 3.0, 2.0, 4.0
    w[(11, 12)], w[(12, 13)], w[(12, 17)] = 1.0, 2.0, 3.0
    delta = np.full(n, 0.5)
    delta[7], delta[12] = 0.6, 0.8
    A = sp.lil_matrix((n, n))
    for (i, j), v in w.items():
        A[i, j] = A[j, i] = -v
    for i in range(n):
        A[i, i] = -A[i].sum() + delta[i]
    return A.tocsr()


def _end_rows(split, f, vertex, pieces):
    """Feature rows of the end at the copy of ``vertex`` in pieces[0] on the line to pieces[1]."""
    for t, (ja, ca, jb, cb) in enumerate(split.vtl):
        for side, (j, c, jt) in enumerate(((ja, ca, jb), (jb, cb, ja))):
            if split.subgraphs[j].vertices[c] == vertex and (j, jt) == pieces:
                return f[2 * t + side]
    raise AssertionError((vertex, pieces))


def test_line_features_hand_computed():
    """Features 1, 4, 5 and 7 by hand from §4 step 3's share rule on a variable-weight split.

    Blocks of 2 on the 5 x 5 grid: four 3 x 3 subgraphs (ids qx + 2 qy), cut lines x = 2, y = 2.
    Edge vertex 7: O = {0, 1}; its edges to 6 (only in 0) and 8 (only in 1) are not split, those to
    2 and 12 (both on the cut line) are halved, delta_7 / 2 per copy:
      copy in 0: 1 + 2/2 + 4/2 + 0.6/2 = 4.3 (off-diagonal sum 4.0), copy in 1: 3 + 1 + 2 + 0.3 = 6.3
      (6.0); 4.3 + 6.3 = a_77 = 10.6.
    Corner 12: O = {0, 1, 2, 3}; each edge lies in two subgraphs (halved), delta_12 / 4 = 0.2:
      copy in 0 (edges to 11, 7): 0.5 + 2 + 0.2 = 2.7; in 1 (13, 7): 1 + 2 + 0.2 = 3.2;
      in 2 (11, 17): 0.5 + 1.5 + 0.2 = 2.2; in 3 (13, 17): 1 + 1.5 + 0.2 = 2.7; sum 10.8 = a_12,12.
    Feature 5 is the twin copy's split weight, feature 4 excludes the copy's own diagonal."""
    A = _hand_grid()
    split = evs.split_grid(A, (5, 5), (2, 2))
    f = features.line_features(split, A)
    ln = np.log
    e = _end_rows(split, f, 7, (0, 1))
    assert np.allclose(e[[0, 1, 2, 3, 4, 5, 6]], [ln(10.6), ln(4.3), ln(2), 1, ln(4.0), ln(6.3), ln(4.0)])
    e = _end_rows(split, f, 7, (1, 0))
    assert np.allclose(e[[1, 4, 5]], [ln(6.3), ln(6.0), ln(4.3)])
    corner = {0: (2.7, 2.5), 1: (3.2, 3.0), 2: (2.2, 2.0), 3: (2.7, 2.5)}
    for (p, q) in [(0, 1), (1, 0), (0, 2), (2, 0), (1, 3), (3, 1), (2, 3), (3, 2)]:
        e = _end_rows(split, f, 12, (p, q))
        assert np.allclose(e[[0, 1, 2, 3, 4, 5]], [ln(10.8), ln(corner[p][0]), ln(4), 2, ln(corner[p][1]),
                                                   ln(corner[q][0])]), (p, q)
    assert np.allclose(f[:, 7], ln(25 / 9))
    # the copies' split weights sum back to a_ii (KCL, App. 2) at every boundary vertex
    for vtx in (7, 12):
        rows = [2 * t + s for t, q in enumerate(split.vtl) for s in (0, 1)
                if split.subgraphs[q[2 * s]].vertices[q[2 * s + 1]] == vtx]
        weights = {}
        for r in rows:
            t, s = divmod(r, 2)
            weights[int(split.vtl[t][2 * s])] = np.exp(f[r, 1])
        assert np.isclose(sum(weights.values()), A[vtx, vtx])


def test_line_features_ragged_subgraph_sizes():
    """Feature 7 = log(n / n_j) with uneven subgraphs: 5 x 4 grid, blocks of 2 -> 3 x 3 and 3 x 2
    subgraphs (9 and 6 copies, n = 20)."""
    dims = (5, 4)
    A = inputs.grid_poisson(dims, sigma=0.7, seed=3)
    split = evs.split_grid(A, dims, (2, 2))
    f = features.line_features(split, A)
    sizes = [len(g.vertices) for g in split.subgraphs]
    assert sorted(sizes) == [6, 6, 9, 9]
    for t, (ja, ca, jb, cb) in enumerate(split.vtl):
        assert np.isclose(f[2 * t, 7], np.log(20 / sizes[ja]))
        assert np.isclose(f[2 * t + 1, 7], np.log(20 / sizes[jb]))
