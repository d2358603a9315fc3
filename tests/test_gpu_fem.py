"""P1 FEM split by elements (uneven subgraphs in RCM order) through the CUDA path vs the oracle."""
import numpy as np
import pytest

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs

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


@pytest.mark.parametrize("precision,nrhs,tol", [("fp64", 1, 1e-12), ("fp64", 16, 1e-12), ("fp32", 16, 5e-4)])
def test_fem_sweeps_match_oracle(vtmlib, precision, nrhs, tol):
    fem, part, osplit = _setup(vtmlib, 3000, 12, seed=5)
    b = inputs.rhs_uniform(fem.A.n, nrhs, seed=5)
    Z = 1e-2
    s = vtmlib.Solver(part, z=Z, precision=precision, nrhs=nrhs)
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


def test_fem_matched_solve(vtmlib):
    fem, part, osplit = _setup(vtmlib, 4000, 16, seed=6)
    b = inputs.rhs_uniform(fem.A.n, 2, seed=6)
    s = vtmlib.Solver(part, z="matched", z_init=1e-2, precision="fp32", nrhs=2)
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=100000)
    As = fem.A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= 1e-8), (rel, st.sweeps)
