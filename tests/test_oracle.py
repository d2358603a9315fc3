"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it follows.  Expected values come from the paper's printed examples
(tests/golden/*.json), closed forms, library routines on tiny inputs, or theorems.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import evs, matching, theory
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from conftest import load_golden


def example_split():
    """The explicit split of Example 4.1 as a SplitGraph (§4, eq. 4.1/4.2)."""
    g = load_golden("example_4_1.json")
    s1 = evs.Subgraph(vertices=np.array(g["vertices_1"]), A=sp.csr_matrix(np.array(g["A1"], float)),
                      share=np.full(4, np.nan), b_explicit=np.array(g["b1"], float))
    s2 = evs.Subgraph(vertices=np.array(g["vertices_2"]), A=sp.csr_matrix(np.array(g["A2"], float)),
                      share=np.full(4, np.nan), b_explicit=np.array(g["b2"], float))
    return evs.SplitGraph(n=6, subgraphs=[s1, s2], vtl=np.array(g["lines"], dtype=np.int64))


def example_system():
    g = load_golden("example_3_1.json")
    return np.array(g["A"], float), np.array(g["b"], float)


# ---------------------------------------------------------------- §4 EVS


def test_example_4_1_sums_back_exactly():
    """App. 2: C_se + C_ju = C, E_se + E_ju = E, f_se + f_ju = f for the printed Example 4.1."""
    A, b = example_system()
    split = example_split()
    assert evs.kcl_residual(split, A) == 0.0
    tot_b = np.zeros(6)
    for j, g in enumerate(split.subgraphs):
        np.add.at(tot_b, g.vertices, split.local_rhs(b, j)[0])
    assert np.array_equal(tot_b, b)


def test_equal_share_rule_on_example_3_1():
    """Our share rule on eq. 3.2 with boundary {V3, V4}: KCL holds, pieces SNND, sources halved."""
    A, b = example_system()
    owners = [(0,), (0,), (0, 1), (0, 1), (1,), (1,)]
    split = evs.split_by_owners(A, owners, [(2, 0, 1), (3, 0, 1)])
    assert evs.kcl_residual(split, A) <= 1e-15 * np.abs(A).max()
    # edge E34 = -2 split in two halves, inner edges untouched (step 3)
    A1 = split.subgraphs[0].A.toarray()
    assert A1[2, 3] == -1.0 and A1[0, 2] == -2.0
    # boundary copy weight: |a31| + |a34|/2 + delta/2 with delta = 8 - 5 = 3
    assert A1[2, 2] == pytest.approx(2.0 + 1.0 + 1.5)
    for g in split.subgraphs:
        assert np.linalg.eigvalsh(g.A.toarray()).min() >= -1e-12
    assert np.allclose(split.local_rhs(b, 0)[0], [1, 2, 1.5, 2.0])


def test_grid_config1_layout():
    """32x32 grid, cut line at 16: pieces 17x17, 16x17, 17x16, 16x16; 62 + 4 lines (Fig. 7 B/C)."""
    A = inputs.grid_poisson((32, 32))
    split = evs.split_grid(A, (32, 32), (16, 16))
    sizes = sorted(len(g.vertices) for g in split.subgraphs)
    assert sizes == [256, 272, 272, 289]
    assert sum(sizes) == 1089
    assert len(split.vtl) == 66
    assert evs.kcl_residual(split, A) <= 4e-16 * np.abs(A.val).max()
    # shares sum to one per vertex
    tot = np.zeros(A.n)
    for g in split.subgraphs:
        np.add.at(tot, g.vertices, g.share)
    assert np.allclose(tot, 1.0, atol=1e-15, rtol=0)


def test_grid_3d_hypercube_counts():
    """Fig. 7 D: a 3D corner vertex has 8 children with 3 lines each (12 lines)."""
    dims, blk = (9, 9, 9), (4, 4, 4)   # 2x2x2 blocks, cut planes at 4
    owners, pairs, nblk = evs.grid_owners(dims, blk)
    assert nblk == (2, 2, 2)
    corner = 4 + 9 * (4 + 9 * 4)
    assert len(owners[corner]) == 8
    assert sum(1 for p in pairs if p[0] == corner) == 12
    edge = 1 + 9 * (4 + 9 * 4)        # on the line y = z = 4
    assert len(owners[edge]) == 4 and sum(1 for p in pairs if p[0] == edge) == 4
    face = 1 + 9 * (1 + 9 * 4)        # on the plane z = 4
    assert len(owners[face]) == 2 and sum(1 for p in pairs if p[0] == face) == 1
    per_copy = {}
    for (i, p, q) in pairs:
        per_copy[(i, p)] = per_copy.get((i, p), 0) + 1
        per_copy[(i, q)] = per_copy.get((i, q), 0) + 1
    assert per_copy[(corner, 0)] == 3


@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_grid_pieces_snnd_and_kcl(sigma):
    """Cor. 4.1: every piece is SNND; KCL up to rounding (variable coefficients)."""
    dims = (7, 6, 5)
    A = inputs.grid_poisson(dims, sigma=sigma, seed=3)
    split = evs.split_grid(A, dims, (3, 3, 2))
    assert evs.kcl_residual(split, A) <= 1e-14 * np.abs(A.val).max()
    for g in split.subgraphs:
        assert np.linalg.eigvalsh(g.A.toarray()).min() >= -1e-12 * np.abs(g.A.data).max()


def test_split_grid_piece_matches_full_split():
    dims = (9, 7, 6)
    A = inputs.grid_poisson(dims, sigma=0.7, seed=5)
    split = evs.split_grid(A, dims, (4, 3, 5))
    for j in range(len(split.subgraphs)):
        v, Aj, share = evs.split_grid_piece(A, dims, (4, 3, 5), j)
        g = split.subgraphs[j]
        assert np.array_equal(v, g.vertices)
        assert abs(Aj - g.A).max() == 0.0
        assert np.array_equal(share, g.share)


def test_not_conformal_rejected():
    """Step 3 needs weak diagonal dominance at the boundary (reading of Cor. 4.1)."""
    A = np.array([[1.0, -2.0, 0], [-2.0, 5.0, -1.0], [0, -1.0, 2.0]])
    with pytest.raises(evs.NotConformal):
        evs.split_by_owners(A, [(0, 1), (1,), (1,)], [(0, 0, 1)])


# ---------------------------------------------------------------- §5 VTM


def test_example_5_1_local_matrices(golden):
    """eq. 5.4 / 5.5: Z3 = 1, Z4 = 0.5 add 1 and 2 to the port diagonals."""
    g = golden("example_5_1.json")
    split = example_split()
    ends = ovtm.ends_of(split, g["Z"])
    assert np.array_equal(ovtm.local_matrix(split, ends, 0).toarray(), np.array(g["K1"]))
    assert np.array_equal(ovtm.local_matrix(split, ends, 1).toarray(), np.array(g["K2"]))


def test_example_5_1_rhs_and_current_update(golden):
    """eq. 5.4 right side 1.6 + x3b - w3b, 1.8 + 2 x4b - w4b and the printed current updates."""
    g = golden("example_5_1.json")
    split = example_split()
    m = ovtm.VTM(split, g["Z"])
    st = m.initial_state()
    rng = np.random.default_rng(0)
    st.u[:] = rng.uniform(-1, 1, st.u.shape)
    st.omega[:] = rng.uniform(-1, 1, st.omega.shape)
    # ends: 0 = 3a, 1 = 3b, 2 = 4a, 3 = 4b
    x3b, w3b, x4b, w4b = st.u[0, 1], st.omega[0, 1], st.u[0, 3], st.omega[0, 3]
    new = m.sweep(st, np.zeros(6))
    rhs = np.array([1, 2, 1.6 + x3b - w3b, 1.8 + 2 * x4b - w4b])
    x1 = np.linalg.solve(np.array(g["K1"], float), rhs)
    assert np.allclose(new.x_local[0][0], x1, rtol=1e-14, atol=1e-14)
    assert new.omega[0, 0] == pytest.approx(-x1[2] + x3b - w3b, abs=1e-14)
    assert new.omega[0, 2] == pytest.approx(-2 * x1[3] + 2 * x4b - w4b, abs=1e-14)


def test_example_5_1_converges_to_direct_solution(golden):
    """Example 5.1 from zero boundary variables converges to the solution of eq. 3.2."""
    g = golden("example_5_1.json")
    A, b = example_system()
    xs = np.linalg.solve(A, b)
    split = example_split()
    m = ovtm.VTM(split, g["Z"])
    st = m.initial_state()
    errs = []
    for k in range(80):
        st = m.sweep(st, b)
        errs.append(ovtm.rms_error(m.assemble(st), xs)[0])
    assert errs[19] < 1e-4
    assert errs[79] < 1e-13
    assert errs[39] < errs[19] < errs[5]


def test_fixed_point_twins_agree_currents_opposite(golden):
    """Thm 4.1 / App. 3 end: at the limit twins have equal potential and opposite currents."""
    g = golden("example_5_1.json")
    A, b = example_system()
    m = ovtm.VTM(example_split(), g["Z"])
    st = m.initial_state()
    for _ in range(120):
        st = m.sweep(st, b)
    u, om = st.u[0], st.omega[0]
    assert np.allclose(u[0::2], u[1::2], atol=1e-13)
    assert np.allclose(om[0::2], -om[1::2], atol=1e-13)


def test_config1_oracle_reaches_1e10():
    """2D Laplacian 32x32, 4 pieces, Z = 1: relative residual 1e-10 and the direct solution."""
    A = inputs.grid_poisson((32, 32))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    split = evs.split_grid(A, (32, 32), (16, 16))
    res = ovtm.solve(split, A, b, 1.0, rtol=1e-10, maxit=2000)
    assert res.history[-1][1] <= 1e-10
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(res.x - xs)) <= 1e-8 * np.max(np.abs(xs))
    assert 100 < res.sweeps < 400


def _owner_split(A, nparts, seed):
    """Random home piece per vertex; a vertex is owned by its home and its neighbours' homes."""
    rng = np.random.default_rng(seed)
    As = A.to_scipy()
    home = rng.integers(0, nparts, A.n)
    # make sure every piece is non-empty
    home[:nparts] = np.arange(nparts)
    owners = []
    for i in range(A.n):
        nb = As.indices[As.indptr[i]:As.indptr[i + 1]]
        owners.append(tuple(sorted(set([int(home[i])]) | set(int(h) for h in home[nb]))))
    pairs = [(i, p, q) for i, o in enumerate(owners) for a, p in enumerate(o) for q in o[a + 1:]]
    return owners, pairs


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_thm_6_1_random_spd_converges(seed):
    """Thm 6.1: SPD A, SNND pieces, any positive Z -> converges to the solution (multilevel too)."""
    A = inputs.random_dd_spd(40, avg_degree=3, excess=0.2, seed=seed)
    owners, pairs = _owner_split(A, 3, seed)
    split = evs.split_by_owners(A.to_scipy(), owners, pairs)
    rng = np.random.default_rng(seed)
    Z = np.exp(rng.uniform(np.log(0.05), np.log(20.0), len(split.vtl)))
    b = inputs.rhs_uniform(A.n, 2, seed=seed)
    res = ovtm.solve(split, A, b, Z, rtol=1e-10, maxit=20000)
    assert res.history[-1][1] <= 1e-10
    xs = ovtm.direct_solve(A, b)
    assert np.allclose(res.x, xs, atol=1e-8 * np.abs(xs).max())


# ---------------------------------------------------------------- §7 matching


def test_example_7_1_input_impedances(golden):
    """Example 7.1: r_in of P3a, P4a, P3b, P4b printed to four decimals (Def. 7.1)."""
    g = golden("example_7_1.json")
    split = example_split()
    A1, A2 = split.subgraphs[0].A, split.subgraphs[1].A
    got = {"3a": matching.input_impedance_open(A1, 2), "4a": matching.input_impedance_open(A1, 3),
           "3b": matching.input_impedance_open(A2, 0), "4b": matching.input_impedance_open(A2, 1)}
    for k, v in g["r_in"].items():
        assert abs(got[k] - v) <= g["tolerance"], (k, got[k], v)


def test_matching_beats_fixed_z_example_5_1(golden):
    """§7.1 (Fig. 11 claim): matched impedances give a much smaller RMS error after 20 sweeps."""
    A, b = example_system()
    xs = np.linalg.solve(A, b)
    split = example_split()
    out = {}
    for name, Z in (("fixed", [1.0, 0.5]), ("matched", matching.matched_impedances(split, terminate=False))):
        m = ovtm.VTM(split, Z)
        st = m.initial_state()
        for _ in range(20):
            st = m.sweep(st, b)
        out[name] = ovtm.rms_error(m.assemble(st), xs)[0]
    assert out["matched"] < 1e-3 * out["fixed"]


def test_terminated_impedance_sherman_morrison():
    """Terminated reading: removing one end's admittance from K_j is a rank-one downdate."""
    A = inputs.grid_poisson((9, 9), sigma=0.5, seed=1)
    split = evs.split_grid(A, (9, 9), (4, 4))
    Z = 0.7
    ends = ovtm.ends_of(split, Z)
    for e in range(0, len(ends.piece), 5):
        j, c = ends.piece[e], ends.local[e]
        K = ovtm.local_matrix(split, ends, j).toarray()
        g = np.linalg.inv(K)[c, c]
        expect = g / (1.0 - g / Z)          # (K - e e^T / Z)^{-1}_cc by Sherman-Morrison
        assert matching.input_impedance_terminated(split, ends, e) == pytest.approx(expect, rel=1e-12)


def test_terminated_equals_open_for_single_port():
    A = inputs.random_dd_spd(9, seed=4).to_dense()
    A = np.diag(np.diag(A)) + np.triu(np.tril(A, 1), -1) - np.diag(np.diag(A))  # tridiagonal part
    A = A + np.diag(np.abs(np.tril(A, -1)).sum(1) + np.abs(np.triu(A, 1)).sum(1) + 0.1)
    owners = [(0,)] * 4 + [(0, 1)] + [(1,)] * 4
    split = evs.split_by_owners(A, owners, [(4, 0, 1)])
    ends = ovtm.ends_of(split, 0.3)
    for e in range(2):
        r_t = matching.input_impedance_terminated(split, ends, e)
        r_o = matching.input_impedance_open(split.subgraphs[ends.piece[e]].A, ends.local[e])
        assert r_t == pytest.approx(r_o, rel=1e-13)


# ---------------------------------------------------------------- App. 3 and §2 closed forms


def _level_one_split(n=30, seed=0):
    A = inputs.random_dd_spd(n, avg_degree=3, excess=0.3, seed=seed)
    As = A.to_scipy()
    home = (np.arange(n) >= n // 2).astype(int)
    owners = []
    for i in range(n):
        nb = As.indices[As.indptr[i]:As.indptr[i + 1]]
        if home[i] == 0 and np.any(home[nb] == 1):
            owners.append((0, 1))
        else:
            owners.append((int(home[i]),))
    pairs = [(i, 0, 1) for i, o in enumerate(owners) if len(o) == 2]
    return A, evs.split_by_owners(As, owners, pairs)


@pytest.mark.parametrize("seed", [0, 1])
def test_a38_operator_reproduces_iteration(seed):
    """eq. A3.8: port errors obey e^k = P e^{k-1} exactly (k >= 2) and rho(P) < 1 (Thm 6.1)."""
    A, split = _level_one_split(seed=seed)
    rng = np.random.default_rng(seed)
    Z = rng.uniform(0.2, 3.0, len(split.vtl))
    P, S, ports = theory.port_operator(split, Z)
    assert np.allclose(S, S.T, atol=1e-12) and np.linalg.eigvalsh(S).min() > 0   # Lemma A3.2
    b = inputs.rhs_uniform(A.n, 1, seed=seed)
    xs = ovtm.direct_solve(A, b)[0]
    m = ovtm.VTM(split, Z)
    st = m.initial_state()
    uhat = lambda s: np.concatenate([s.u[0, 0::2], s.u[0, 1::2]])
    ustar = np.array([xs[split.subgraphs[j].vertices[c]] for j, c in ports])
    st = m.sweep(st, b)
    prev = uhat(st) - ustar
    for k in range(2, 12):
        st = m.sweep(st, b)
        cur = uhat(st) - ustar
        assert np.linalg.norm(cur - P @ prev) <= 1e-10 * np.linalg.norm(prev)
        prev = cur
    assert theory.spectral_radius(P) < 1.0


def _chain_split(n=9, split_at=4, seed=3):
    rng = np.random.default_rng(seed)
    off = -rng.uniform(0.3, 1.0, n - 1)
    A = np.diag(np.r_[0, np.abs(off)] + np.r_[np.abs(off), 0] + rng.uniform(0.05, 0.5, n))
    A += np.diag(off, 1) + np.diag(off, -1)
    owners = [(0,)] * split_at + [(0, 1)] + [(1,)] * (n - split_at - 1)
    return A, evs.split_by_owners(A, owners, [(split_at, 0, 1)])


def test_single_line_reflection_rate():
    """§2 eq. 2.1 with Def. 7.1: wave errors contract by Gamma_a Gamma_b every two sweeps."""
    A, split = _chain_split()
    b = np.linspace(-1, 1, A.shape[0])
    Z = 0.37
    ra = matching.input_impedance_open(split.subgraphs[0].A, split.vtl[0, 1])
    rb = matching.input_impedance_open(split.subgraphs[1].A, split.vtl[0, 3])
    ga, gb = theory.reflection_coefficient(ra, Z), theory.reflection_coefficient(rb, Z)
    m = ovtm.VTM(split, Z)
    st = m.initial_state()
    waves = []
    for _ in range(600):
        st = m.sweep(st, b)
        waves.append(m.waves_out(st)[0].copy())
    wstar = waves[-1]
    assert abs(ga * gb) < 0.97
    e = [w - wstar for w in waves]
    for k in range(2, 12):
        assert e[k + 2][0] == pytest.approx(ga * gb * e[k][0], rel=1e-9, abs=1e-15)


def test_matched_line_exact_in_three_sweeps():
    """Gamma_b = 0 (Z = r_in of side b): exact after three sweeps from zero."""
    A, split = _chain_split(n=11, split_at=6, seed=7)
    b = np.cos(np.arange(A.shape[0]))
    rb = matching.input_impedance_open(split.subgraphs[1].A, split.vtl[0, 3])
    xs = np.linalg.solve(A, b)
    m = ovtm.VTM(split, rb)
    st = m.initial_state()
    for k in range(1, 4):
        st = m.sweep(st, b)
        err = np.max(np.abs(m.assemble(st)[0] - xs))
        if k < 3:
            assert err > 1e-6
    assert err < 1e-13
