"""P1 FEM split by elements (uneven subgraphs in RCM order) through the CUDA path vs the oracle."""
import numpy as np
import pytest

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from test_precision_bounds import TOL_FP16, TOL_FP32  # noqa: F401

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _setup(vtmlib, npts, parts, seed):
    fem = inputs.fem_delaunay(npts, seed=seed)
    part = vtmlib.partition_evs(fem.A, "elements", elements=dict(elem_nodes=fem.elem_nodes, elem_mats=fem.elem_mats,
                                                               node_unknown=fem.node_unknown,
                                                               elem_coords=fem.centroids), npieces=parts)
    osplit = evs.split_by_elements(fem.A, fem.elem_nodes, fem.elem_mats, fem.node_unknown,
                                   evs.rcb(fem.centroids, parts))
    return fem, part, osplit


def _maps(part, osplit):
    """Library copy order -> oracle copy order, library end order -> oracle end order."""
    offs = np.cumsum([0] + [len(g.vertices) for g in osplit.subgraphs])
    cmap = []
    for j in range(part.info().npieces):
        v = part.piece(j)[0]
        pos = np.searchsorted(osplit.subgraphs[j].vertices, v)
        cmap.append(offs[j] + pos)
    cmap = np.concatenate(cmap)
    idx = {}
    for t, (p, c, q, d) in enumerate(osplit.vtl):
        idx[(int(osplit.subgraphs[p].vertices[c]), int(p), int(q))] = t
    emap = []
    for (pa, la, pb, lb) in part.lines():
        v = int(part.piece(int(pa))[0][la])
        t = idx[(v, int(pa), int(pb))]
        emap += [2 * t, 2 * t + 1]
    return cmap, np.array(emap)


@pytest.mark.parametrize("precision,nrhs,tol", [("fp64", 1, 1e-12), ("fp64", 16, 1e-12), ("fp32", 16, TOL_FP32)])
def test_fem_sweeps_match_oracle(vtmlib, precision, nrhs, tol):
    fem, part, osplit = _setup(vtmlib, 3000, 12, seed=5)
    b = inputs.rhs_uniform(fem.A.n, nrhs, seed=5)
    Z = 1e-2
    s = vtmlib.Solver(part, z=Z, precision=precision, nrhs=nrhs, form="band")
    s.set_rhs(b)
    s.reset()
    s.iterate(3)
    m = ovtm.VTM(osplit, Z)
    st = m.initial_state(nrhs)
    for _ in range(3):
        st = m.sweep(st, b)
    ref_c = np.concatenate(st.x_local, axis=1)
    cmap, emap = _maps(part, osplit)
    got = s.copies()
    assert np.max(np.abs(got - ref_c[:, cmap])) <= tol * np.max(np.abs(ref_c))
    w = m.waves_out(st)[:, emap]
    assert np.max(np.abs(s.get_state() - w)) <= tol * np.max(np.abs(w))


@pytest.mark.parametrize("nrhs", [2, 16])
def test_fem_scaled_impedance_solve(vtmlib, nrhs):
    """FP32 sweeps with FP64 defect correction on the 1e-3/1e3 checkerboard: impedances scaled by the
    two copies' split weights, Z_t = 6 / (d_a + d_b), reach 1e-8 (uniform and matched impedances do
    not converge usefully at this contrast; checked with the oracle)."""
    fem, part, osplit = _setup(vtmlib, 4000, 16, seed=6)
    f = part.line_features()
    d = np.exp(f[:, 1].astype(np.float64))
    Z = 6.0 / (d[0::2] + d[1::2])
    b = inputs.rhs_uniform(fem.A.n, nrhs, seed=6)
    s = vtmlib.Solver(part, z=Z, precision="fp32", nrhs=nrhs)
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=100000)
    As = fem.A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= 1e-8), (rel, st.sweeps, s.info().flagged_pieces)


@pytest.mark.parametrize("nrhs", [1, 16])
def test_fem_flagged_subgraphs_match_fp64(vtmlib, nrhs):
    """Nearly floating subgraphs (Z = 1e4: 1/Z is 1e-7 of the stiff coefficient) lose their FP32
    digits; the factorisation flags them and they are factored and swept in FP64 (for 16 right-hand
    sides the forward result of those subgraphs is kept in FP64 between the two passes).  After one
    sweep from zero waves (subgraphs independent) the flagged subgraphs agree with the FP64 solver
    to the FP32 rounding of their sources and outputs."""
    fem, part, osplit = _setup(vtmlib, 6000, 24, seed=9)
    b = inputs.rhs_uniform(fem.A.n, nrhs, seed=9)
    s32 = vtmlib.Solver(part, z=1e4, precision="fp32", nrhs=nrhs)
    s64 = vtmlib.Solver(part, z=1e4, precision="fp64", nrhs=nrhs)
    for s in (s32, s64):
        s.set_rhs(b)
        s.reset()
        s.iterate(1)
    bits = s32.piece_precision()
    assert s32.info().flagged_pieces == int(np.sum(bits == 64)) >= 1
    assert np.all(s64.piece_precision() == 64)
    x32, x64 = s32.copies(), s64.copies()
    offs = np.cumsum([0] + [part.piece(j)[0].size for j in range(part.info().npieces)])
    for j in np.nonzero(bits == 64)[0]:
        a, c = x32[:, offs[j]:offs[j + 1]], x64[:, offs[j]:offs[j + 1]]
        assert np.max(np.abs(a - c)) <= 1e-5 * np.max(np.abs(c)), j
