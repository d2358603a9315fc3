"""The learned-impedance perceptron kernels and the impedance modes against the FP64 oracle (GPU).

Tolerances: the kernels compute in FP32 with BF16 weights; the oracle uses the same BF16-rounded
weights in FP64, so outputs and gradients agree to FP32 accumulation error (1e-4 relative to the
largest value); impedances from the input-impedance rule agree to 1e-10 in FP64.
"""
import numpy as np
import pytest

from oracle import evs, features, matching, mlp as omlp
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1.5, (n, 8)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.3 * X[:, 1] * X[:, 2] - 0.2 * X[:, 3]).astype(np.float32)
    return X, t


def test_forward_and_gradient_match_oracle(vtmlib):
    m = vtmlib.MLP(seed=7)
    p = m.get_params()
    X, t = _data(1000, 0)       # 1000 = several 128-sample tiles and a ragged tail
    Xd, td = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    y = torch.empty(len(X), device="cuda")
    m.forward(Xd, y)
    torch.cuda.synchronize()
    pb = omlp.bf16_round(p)
    yref, _ = omlp.forward(pb, X)
    assert np.max(np.abs(y.cpu().numpy() - yref)) <= 1e-4 * np.max(np.abs(yref))
    loss = m.loss_grad(Xd, td)
    lref, gref = omlp.loss_and_grad(pb, X, t)
    assert abs(loss - lref) <= 1e-4 * lref
    g = m.get_grads()
    assert np.max(np.abs(g - gref)) <= 1e-4 * np.max(np.abs(gref))


def test_adam_matches_oracle_trajectory(vtmlib):
    m = vtmlib.MLP(seed=3)
    p = m.get_params().astype(np.float64)
    X, t = _data(384, 1)
    Xd, td = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    mo, vo = np.zeros_like(p), np.zeros_like(p)
    for k in range(1, 4):
        m.loss_grad(Xd, td)
        m.adam_step(lr=1e-3)
        _, g = omlp.loss_and_grad(omlp.bf16_round(p.astype(np.float32)), X, t)
        p, mo, vo = omlp.adam_step(p, mo, vo, g, k, lr=1e-3)
    got = m.get_params()
    # Adam normalises each step to ~lr, so the FP32/FP64 gradient difference shows only where
    # |g| is tiny; compare the displacement from the start with a small absolute tolerance
    assert np.max(np.abs(got - p)) <= 2e-4


def test_training_reduces_loss(vtmlib):
    m = vtmlib.MLP(seed=11)
    X, t = _data(4096, 2)
    Xd, td = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    first = m.loss_grad(Xd, td)
    for _ in range(300):
        m.loss_grad(Xd, td)
        m.adam_step(lr=3e-3)
    assert m.loss_grad(Xd, td) < 0.2 * first


def test_learned_mode_uses_the_model(vtmlib):
    dims, block = (20, 18), (8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=5)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    m = vtmlib.MLP(seed=5)
    s = vtmlib.Solver(part, z=m, precision="fp64")
    z = s.impedances()
    osplit = evs.split_grid(A, dims, block)
    f = features.line_features(osplit, A)
    yo, _ = omlp.forward(omlp.bf16_round(m.get_params()), f)
    zo = np.exp(0.5 * (yo[0::2] + yo[1::2]))
    idx = {tuple(int(x) for x in q): t for t, q in enumerate(osplit.vtl)}
    order = [idx[tuple(int(x) for x in q)] for q in part.lines()]
    assert np.max(np.abs(np.log(z) - np.log(zo[order]))) <= 1e-4


def test_input_impedances_and_matched_mode(vtmlib):
    dims, block = (13, 11), (4, 5)
    A = inputs.grid_poisson(dims, sigma=0.8, seed=6)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    idx = {tuple(int(x) for x in q): t for t, q in enumerate(osplit.vtl)}
    order = [idx[tuple(int(x) for x in q)] for q in part.lines()]
    s = vtmlib.Solver(part, z=0.7, precision="fp64", nrhs=4)
    r = s.input_impedances()
    ends = ovtm.ends_of(osplit, 0.7)
    rref = np.array([matching.input_impedance_terminated(osplit, ends, e) for e in range(len(ends.piece))])
    eo = np.ravel([[2 * t, 2 * t + 1] for t in order])
    assert np.max(np.abs(r - rref[eo]) / rref[eo]) <= 1e-10
    sm = vtmlib.Solver(part, z="matched", z_init=0.7, precision="fp64")
    zref = matching.matched_impedances(osplit, Z0=0.7, terminate=True)
    assert np.max(np.abs(sm.impedances() - zref[order]) / zref[order]) <= 1e-10
