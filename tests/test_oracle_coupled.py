"""Pins of the coupled-line oracle (oracle/coupled.py, §7.2, Thm 7.1) against facts that do not
come from the oracle itself: the uncoupled oracle as the special case Y = diag(1/Z), the direct
solution (Thm 7.1), Thm 4.1 at the fixed point, the multi-conductor reflection law of a bundle
and the matched bundle that is exact after three sweeps."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coupled, evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def _grid(dims, block, sigma=0.0, seed=3):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=seed)
    return A, evs.split_grid(A, dims, block)


def _run(m, b, k):
    st = m.initial_state(np.atleast_2d(b).shape[0])
    for _ in range(k):
        st = m.sweep(st, b)
    return st


def test_diagonal_admittance_is_the_uncoupled_oracle():
    """Y = diag(1/Z_t): the same iteration as Table 1 with scalar impedances (multilevel corner
    lines included)."""
    A, split = _grid((32, 32), (16, 16), sigma=0.8)
    b = inputs.rhs_uniform(A.n, 2, seed=1)
    Z = np.random.default_rng(0).uniform(0.3, 3.0, len(split.vtl))
    m0, m1 = ovtm.VTM(split, Z), coupled.CoupledVTM(split, sp.diags(1.0 / Z))
    s0, s1 = _run(m0, b, 9), _run(m1, b, 9)
    w0 = m0.waves_out(s0)
    assert np.max(np.abs(m1.waves_out(s1) - w0)) <= 1e-12 * np.max(np.abs(w0))
    assert np.max(np.abs(m1.assemble(s1) - m0.assemble(s0))) <= 1e-12


def _random_bundle_admittance(split, rng):
    """Block diagonal over bundles: diag(1/Z) plus a random dense SPD block per bundle."""
    m = len(split.vtl)
    Y = sp.lil_matrix((m, m))
    for ts in coupled.bundles(split).values():
        B = rng.normal(size=(len(ts), len(ts)))
        blk = 0.3 * B @ B.T / len(ts) + np.diag(rng.uniform(0.2, 2.0, len(ts)))
        Y[np.ix_(ts, ts)] = 0.5 * (blk + blk.T)
    return Y.tocsr()


@pytest.mark.parametrize("dims,block,sigma", [((20, 20), (7, 7), 1.0), ((9, 8, 7), (4, 4, 4), 0.5)])
def test_theorem_7_1_random_spd_bundles_converge(dims, block, sigma):
    """Thm 7.1: with every Z_j SPD the iteration converges to the solution of A x = b."""
    A, split = _grid(dims, block, sigma)
    b = inputs.rhs_uniform(A.n, 1, seed=2)
    m = coupled.CoupledVTM(split, _random_bundle_admittance(split, np.random.default_rng(5)))
    st = m.initial_state()
    for k in range(1, 3001):
        st = m.sweep(st, b)
        if k % 20 == 0 and ovtm.relative_residual(A, b, m.assemble(st))[0] <= 1e-11:
            break
    assert ovtm.relative_residual(A, b, m.assemble(st))[0] <= 1e-11
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(m.assemble(st) - xs)) <= 1e-8 * np.max(np.abs(xs))
    # Thm 4.1 at the fixed point: twin potentials agree, inflow currents are opposite
    e = np.arange(len(m.end_piece))
    scale = np.max(np.abs(st.u))
    assert np.max(np.abs(st.u[:, e] - st.u[:, e ^ 1])) <= 1e-8 * scale
    assert np.max(np.abs(st.omega[:, e] + st.omega[:, e ^ 1])) <= 1e-8 * max(1.0, np.max(np.abs(st.omega)))


def test_admittance_checks():
    A, split = _grid((12, 12), (4, 4))
    pairs, w = coupled.adjacent_line_pairs(split, A)
    Y = coupled.laplacian_admittance(split, 1.5, pairs, 0.7 * w)
    assert abs(Y - Y.T).max() == 0
    assert np.linalg.eigvalsh(Y.toarray()).min() > 0
    # every pair joins two lines of one bundle whose copies are neighbours on both sides
    key = {int(t): k for k, ts in coupled.bundles(split).items() for t in ts}
    for t, u in pairs:
        assert key[int(t)] == key[int(u)]
    # a coupling across bundles is not a bundle impedance
    bad = sp.lil_matrix(sp.diags(np.ones(len(split.vtl))))
    t0 = 0
    u0 = next(u for u in range(len(split.vtl)) if key[u] != key[t0])
    bad[t0, u0] = bad[u0, t0] = -0.1
    with pytest.raises(ValueError):
        coupled.CoupledVTM(split, bad.tocsr())


def _two_pieces(sigma=0.6):
    """A 2D grid cut once: two subgraphs, both touching the Dirichlet boundary (Ã_j nonsingular),
    one bundle of 17 lines."""
    A, split = _grid((18, 17), (9, 16), sigma, seed=7)
    assert len(split.subgraphs) == 2 and len(coupled.bundles(split)) == 1
    return A, split


def _input_impedance_matrix(split, j, ends):
    """R_j = P^T Ã_j^{-1} P over the bundle, in line order (Def. 7.1 for all lines at once; the
    other subgraph is absent, so nothing else is terminated)."""
    Aj = split.subgraphs[j].A.toarray()
    P = np.zeros((Aj.shape[0], len(ends)))
    P[ends, np.arange(len(ends))] = 1.0
    return P.T @ np.linalg.solve(Aj, P)


def _sides(split):
    """Local copy at subgraph 0 and 1 of every line, and the end ids at each side."""
    v = split.vtl
    ea = np.where(v[:, 0] == 0, 2 * np.arange(len(v)), 2 * np.arange(len(v)) + 1)
    la = np.where(v[:, 0] == 0, v[:, 1], v[:, 3])
    lb = np.where(v[:, 0] == 0, v[:, 3], v[:, 1])
    return ea, ea ^ 1, la, lb


def test_bundle_reflection_law():
    """Microwave-network closed form: the wave error leaving subgraph a is
    Gamma_a = (R_a - Z)(R_a + Z)^{-1} times the error that arrived there, with the bundle's full
    impedance matrix Z = Y^{-1} and R_a the bundle's input impedance matrix."""
    A, split = _two_pieces()
    pairs, w = coupled.adjacent_line_pairs(split, A)
    Y = coupled.laplacian_admittance(split, np.linspace(0.5, 2.0, len(split.vtl)), pairs, 0.8 * w)
    m = coupled.CoupledVTM(split, Y)
    ea, eb, la, lb = _sides(split)
    Z = np.linalg.inv(Y.toarray())
    gam = {}
    for side, loc in ((0, la), (1, lb)):
        R = _input_impedance_matrix(split, side, loc)
        gam[side] = (R - Z) @ np.linalg.inv(R + Z)
    b = inputs.rhs_uniform(A.n, 1, seed=4)
    st = m.initial_state()
    ws = []
    for _ in range(400):
        st = m.sweep(st, b)
        ws.append(m.waves_out(st)[0])
    assert ovtm.relative_residual(A, b, m.assemble(st))[0] <= 1e-12   # ws[-1] is the fixed point
    wstar = ws[-1]
    for k in range(1, 6):
        da1, db0 = ws[k][ea] - wstar[ea], ws[k - 1][eb] - wstar[eb]
        db1, da0 = ws[k][eb] - wstar[eb], ws[k - 1][ea] - wstar[ea]
        assert np.linalg.norm(da1 - gam[0] @ db0) <= 1e-9 * np.linalg.norm(db0)
        assert np.linalg.norm(db1 - gam[1] @ da0) <= 1e-9 * np.linalg.norm(da0)


def test_matched_bundle_is_exact_after_three_sweeps():
    """Z = R_a (the full input impedance matrix of subgraph a) makes Gamma_a = 0: a's outgoing
    wave is its open-circuit potential from the first sweep on, b is exact at sweep 2 and a at
    sweep 3."""
    A, split = _two_pieces()
    ea, eb, la, lb = _sides(split)
    Ra = _input_impedance_matrix(split, 0, la)
    Y = np.linalg.inv(Ra)
    Y = 0.5 * (Y + Y.T)
    m = coupled.CoupledVTM(split, sp.csr_matrix(Y))
    b = inputs.rhs_uniform(A.n, 1, seed=9)
    res = []
    st = m.initial_state()
    for _ in range(3):
        st = m.sweep(st, b)
        res.append(ovtm.relative_residual(A, b, m.assemble(st))[0])
    assert res[1] > 1e-6 and res[2] <= 1e-11
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(m.assemble(st) - xs)) <= 1e-10 * np.max(np.abs(xs))


def _sweeps_to(m, A, b, rtol, maxit=2000):
    st = m.initial_state()
    for k in range(1, maxit + 1):
        st = m.sweep(st, b)
        if k % 5 == 0 and ovtm.relative_residual(A, b, m.assemble(st))[0] <= rtol:
            return k
    return maxit


def test_tangential_coupling_reduces_sweeps():
    """The outcome that motivates §7.2's coupling (not a pin of the arithmetic): a conductance
    between neighbouring lines of a bundle, proportional to the local edge weight, lets a larger
    Z damp the smooth interface modes without slowing the rough ones; on a 4 x 4 split of a 2D
    Laplacian the coupled lines need well under 60 % of the sweeps of the best uniform Z."""
    A, split = _grid((48, 48), (12, 12))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    best = min(_sweeps_to(ovtm.VTM(split, z), A, b, 1e-8) for z in (1.0, 2.0, 4.0))
    pairs, w = coupled.adjacent_line_pairs(split, A)
    cpl = _sweeps_to(coupled.CoupledVTM(split, coupled.laplacian_admittance(split, 8.0, pairs, 0.25 * w)), A, b, 1e-8)
    assert cpl < 0.6 * best
