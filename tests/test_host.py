"""Host-side logic of the C-ABI library on CPU: exports, EVS partition parity with the oracle.

vtm_partition_evs runs on the host only (no device crossing), so its split is compared here with
the oracle's independent split, element by element.
"""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import evs
from paper_0807_1949_gb300 import inputs
from conftest import ROOT


def test_library_exports_every_declared_symbol(vtmlib):
    hdr = open(os.path.join(ROOT, "include", "vtm.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(vtm_\w+)\s*\(", hdr, re.M))
    assert {"vtm_partition_evs", "vtm_setup", "vtm_iterate", "vtm_solve"} <= declared
    lib = vtmlib._lib
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert vtmlib.version() == 1


def _local_dense(piece):
    v, s, (rp, col, val) = piece
    m = len(v)
    return v, s, sp.csr_matrix((val, col, rp), shape=(m, m)).toarray()


def _compare_split(part, osplit, atol=0.0):
    info = part.info()
    assert info.npieces == len(osplit.subgraphs)
    for j, g in enumerate(osplit.subgraphs):
        v, s, Aj = _local_dense(part.piece(j))
        assert np.array_equal(v, g.vertices)
        assert np.array_equal(s, g.share)
        ref = g.A.toarray()
        assert np.max(np.abs(Aj - ref)) <= atol * max(1.0, np.abs(ref).max()), j
    lines = {tuple(q) for q in part.lines()}
    olines = {tuple(int(x) for x in q) for q in osplit.vtl}
    assert lines == olines


def test_grid_config1_partition_matches_oracle(vtmlib):
    A = inputs.grid_poisson((32, 32))
    part = vtmlib.partition_evs(A, "grid", dims=(32, 32), block=(16, 16))
    info = part.info()
    assert (info.npieces, info.ncopies, info.nlines) == (4, 1089, 66)
    _compare_split(part, evs.split_grid(A, (32, 32), (16, 16)), atol=0.0)


@pytest.mark.parametrize("dims,block,sigma", [((9, 7, 6), (4, 3, 5), 0.7), ((10, 9, 9), (4, 4, 4), 1.5),
                                               ((17, 5), (4, 2), 1.0), ((5, 5, 5), (2, 2, 2), 0.0)])
def test_grid_partition_matches_oracle(vtmlib, dims, block, sigma):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=11)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    _compare_split(part, evs.split_grid(A, dims, block), atol=1e-15)


def test_owner_partition_matches_oracle(vtmlib):
    A = inputs.random_dd_spd(60, avg_degree=4, excess=0.2, seed=2)
    rng = np.random.default_rng(2)
    As = A.to_scipy()
    home = rng.integers(0, 4, A.n)
    home[:4] = np.arange(4)
    owners = [tuple(sorted({int(home[i])} | {int(h) for h in home[As.indices[As.indptr[i]:As.indptr[i + 1]]]}))
              for i in range(A.n)]
    lines = [(i, p, q) for i, o in enumerate(owners) for a, p in enumerate(o) for q in o[a + 1:]]
    part = vtmlib.partition_evs(A, "owners", owners=owners, lines=lines)
    _compare_split(part, evs.split_by_owners(As, owners, lines), atol=1e-15)


def example_explicit(golden):
    g = golden("example_4_1.json")
    gb = golden("example_3_1.json")
    A = inputs.csr_from_dense(np.array(gb["A"], float))
    b = np.array(gb["b"], float)
    A1, A2 = sp.csr_matrix(np.array(g["A1"], float)), sp.csr_matrix(np.array(g["A2"], float))
    blk = sp.block_diag([A1, A2]).tocsr()
    # local columns: the block-diagonal column minus the piece's first copy
    cols = blk.indices.copy()
    cols[blk.indptr[4]:] -= 4
    verts = np.array(g["vertices_1"] + g["vertices_2"])
    share = np.concatenate([np.array(g["b1"]), np.array(g["b2"])]) / b[verts]
    la = [4 * l[0] + l[1] for l in g["lines"]]
    lb = [4 * l[2] + l[3] for l in g["lines"]]
    spec = dict(piece_ptr=[0, 4, 8], copy_vertex=verts, copy_share=share, local_rowptr=blk.indptr,
                local_col=cols, local_val=blk.data, line_copy_a=la, line_copy_b=lb)
    return A, b, spec


def test_explicit_partition_example_4_1(vtmlib, golden):
    A, b, spec = example_explicit(golden)
    part = vtmlib.partition_evs(A, "explicit", explicit=spec)
    info = part.info()
    assert (info.npieces, info.ncopies, info.nlines, info.nboundary) == (2, 8, 2, 2)
    g = golden("example_4_1.json")
    assert np.array_equal(_local_dense(part.piece(0))[2], np.array(g["A1"]))
    assert np.array_equal(_local_dense(part.piece(1))[2], np.array(g["A2"]))


def test_errors_are_reported(vtmlib):
    A = inputs.grid_poisson((6, 6))
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(A, "grid", dims=(6, 5), block=(3, 3))
    assert e.value.code == 1
    # not symmetric
    bad = inputs.CSR(n=A.n, rowptr=A.rowptr, col=A.col, val=A.val.copy())
    bad.val[1] *= 2
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(bad, "grid", dims=(6, 6), block=(3, 3))
    assert e.value.code == 2
    # not conformal at a boundary vertex
    D = np.array([[1.0, -2.0, 0], [-2.0, 5.0, -1.0], [0, -1.0, 2.0]])
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(inputs.csr_from_dense(D), "owners", owners=[(0, 1), (1,), (1,)], lines=[(0, 0, 1)])
    assert e.value.code == 3


def test_malformed_rowptr_is_an_error_before_any_partner_lookup(vtmlib):
    """Row 19 of a 6 x 6 grid made to end before it starts: row 14's symmetric partner, row 20,
    would be read through that range; the library reports the bad row pointer instead."""
    A = inputs.grid_poisson((6, 6))
    rp = A.rowptr.copy()
    rp[20] = rp[19] - 1
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(inputs.CSR(n=A.n, rowptr=rp, col=A.col, val=A.val), "grid", dims=(6, 6), block=(3, 3))
    assert e.value.code == 1 and "monotone" in str(e.value)


def test_first_error_of_a_threaded_matrix_check(vtmlib):
    """1024^2 rows (checked in 64 blocks on the host threads) with two defects: a column index out of
    range in row 100 and an unsymmetric value in row 900000; the error of row 100 is reported, as
    from one loop over the rows."""
    A = inputs.grid_poisson((1024, 1024))
    col, val = A.col.copy(), A.val.copy()
    col[A.rowptr[101] - 1] = A.n + 5
    val[A.rowptr[900000]] *= 2
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(inputs.CSR(n=A.n, rowptr=A.rowptr, col=col, val=val), "grid", dims=(1024, 1024),
                             block=(512, 512))
    assert e.value.code == 1 and "out of range" in str(e.value)
    val2 = A.val.copy()
    val2[A.rowptr[900000]] *= 2
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(inputs.CSR(n=A.n, rowptr=A.rowptr, col=A.col, val=val2), "grid", dims=(1024, 1024),
                             block=(512, 512))
    assert e.value.code == 2


@pytest.mark.parametrize("dims,block,sigma", [((9, 7, 6), (4, 3, 5), 0.7), ((17, 12), (8, 5), 1.3)])
def test_line_features_match_oracle(vtmlib, dims, block, sigma):
    from oracle import features
    A = inputs.grid_poisson(dims, sigma=sigma, seed=3)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    got = part.line_features()
    ref = features.line_features(osplit, A)
    idx = {tuple(int(x) for x in q): t for t, q in enumerate(osplit.vtl)}
    order = []
    for q in part.lines():
        t = idx[tuple(int(x) for x in q)]
        order += [2 * t, 2 * t + 1]
    assert np.allclose(got, ref[order], rtol=1e-6, atol=1e-6)


@pytest.fixture(scope="module")
def threaded_split(vtmlib):
    """65^3 in 4^3 blocks: 288,000 lines (576,000 ends), enough for the library to spread the lines
    and ends over its host threads (it does so from 64 blocks of 4096); the library's partition
    and the oracle's split of the same matrix."""
    dims, block = (65, 65, 65), (4, 4, 4)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=5)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    assert len(osplit.vtl) >= 64 * 4096
    return A, part, osplit


def test_line_features_match_oracle_on_a_threaded_partition(threaded_split):
    """2000 random lines (4000 ends) of the threaded partition against the oracle."""
    from oracle import features
    A, part, osplit = threaded_split
    got = part.line_features()
    assert got.shape == (2 * len(osplit.vtl), 8)
    pos = {tuple(int(x) for x in q): t for t, q in enumerate(part.lines())}
    rng = np.random.default_rng(11)
    pick = rng.choice(len(osplit.vtl), size=2000, replace=False)
    ref = features.line_features(osplit, A, lines=pick)
    rows = []
    for t in pick:
        u = pos[tuple(int(x) for x in osplit.vtl[t])]
        rows += [2 * u, 2 * u + 1]
    assert np.allclose(got[rows], ref, rtol=1e-6, atol=1e-6)


def test_line_pairs_match_oracle_on_a_threaded_partition(threaded_split):
    """The candidate couplings of the threaded partition: the oracle's set of pairs with |a_ik|,
    listed in increasing order of the first line as from one loop over the lines."""
    from oracle import coupled
    A, part, osplit = threaded_split
    pr, w = part.line_pairs()
    opr, ow = coupled.adjacent_line_pairs(osplit, A)
    assert len(pr) == len(opr) > 0
    q, oq = part.lines(), osplit.vtl
    got = {frozenset((tuple(q[t]), tuple(q[u]))): x for (t, u), x in zip(pr, w)}
    ref = {frozenset((tuple(int(v) for v in oq[t]), tuple(int(v) for v in oq[u]))): x for (t, u), x in zip(opr, ow)}
    assert got.keys() == ref.keys()
    assert all(got[k] == ref[k] for k in ref)
    assert np.all(pr[:, 0] < pr[:, 1]) and np.all(np.diff(pr[:, 0]) >= 0)


def test_rcb_is_identical_to_oracle(vtmlib):
    rng = np.random.default_rng(0)
    for dim, n, parts in [(2, 5000, 37), (3, 3000, 64), (2, 999, 2)]:
        pts = rng.uniform(size=(n, dim))
        pts[:50] = pts[0]  # ties broken by id
        assert np.array_equal(vtmlib.rcb(pts, parts), evs.rcb(pts, parts))


def test_element_partition_matches_oracle(vtmlib):
    """P1 FEM split by elements (RCB of centroids): pieces, shares and lines against the oracle;
    the pieces sum back to A (KCL) and are SNND."""
    fem = inputs.fem_delaunay(600, seed=3)
    A = fem.A
    parts = 9
    part = vtmlib.partition_evs(A, "elements", elements=dict(elem_nodes=fem.elem_nodes, elem_mats=fem.elem_mats,
                                                           node_unknown=fem.node_unknown, elem_coords=fem.centroids),
                                npieces=parts)
    ep = evs.rcb(fem.centroids, parts)
    osplit = evs.split_by_elements(A, fem.elem_nodes, fem.elem_mats, fem.node_unknown, ep)
    info = part.info()
    assert info.npieces == parts and info.nlines == len(osplit.vtl)
    assert evs.kcl_residual(osplit, A) <= 1e-12 * np.abs(A.val).max()
    for j, g in enumerate(osplit.subgraphs):
        v, s, Aj = _local_dense(part.piece(j))
        order = np.argsort(v)                       # library order is RCM; compare by vertex
        assert np.array_equal(v[order], g.vertices)
        assert np.allclose(s[order], g.share, rtol=0, atol=0)
        ref = g.A.toarray()
        assert np.max(np.abs(Aj[np.ix_(order, order)] - ref)) <= 1e-12 * np.abs(ref).max()
        assert np.linalg.eigvalsh(ref).min() >= -1e-9 * np.abs(ref).max()
    lines = set()
    for (pa, la, pb, lb) in part.lines():
        va = part.piece(int(pa))[0][la]
        lines.add((int(va), int(pa), int(pb)))
    olines = {(int(osplit.subgraphs[p].vertices[c]), int(p), int(q)) for (p, c, q, _) in osplit.vtl}
    assert lines == olines


def test_committed_models_are_well_formed():
    import json
    import os
    from paper_0807_1949_gb300 import learned_z
    for name in ("z_poisson2d-256.json", "z_poisson3d.json", "z_poisson3d-wide.json"):
        with open(os.path.join(learned_z.MODELS, name)) as f:
            d = json.load(f)
        p = np.asarray(d["params"])
        assert p.shape == (4801,) and np.all(np.isfinite(p))
        ms = d["median_sweeps"]
        assert ms["learned"] < ms["z1"] and ms["learned"] < ms.get("matched", np.inf)
        # the coupled-line rule selected on held-out seeds, and its gain on the test seeds
        c = d["coupling"]
        assert c["z_scale"] > 0 and c["gamma"] > 0 and c["select_seeds"] >= 1
        assert c["median_sweeps"]["coupled"] < c["median_sweeps"]["learned"]
        assert 8 <= len(c["eval"]) <= d["test_seeds"]


def test_profiled_search_records():
    """The recorded GPU comparison of the plain and the profiled search walks (held-out seeds of the
    2D family) and the network trained on profiled-walk targets, evaluated on the same seeds."""
    import json
    import os
    from paper_0807_1949_gb300 import learned_z
    with open(os.path.join(learned_z.MODELS, "z_poisson2d-256.json")) as f:
        shipped = json.load(f)
    with open(os.path.join(learned_z.MODELS, "z_poisson2d-256-profiled.json")) as f:
        prof = json.load(f)
    p = np.asarray(prof["params"])
    assert p.shape == (4801,) and np.all(np.isfinite(p))
    assert prof["search_walk"] == "profiled" and len(prof["search"]) == prof["train_seeds"] == 24
    cmp_rows = {r["seed"]: r for r in shipped["search_compare"]["rows"]}
    assert len(cmp_rows) == 8
    # per problem, the profiled walk's own family impedances against the plain walk's
    ratio = [r["profiled"]["sweeps"] / r["plain"]["sweeps"] for r in cmp_rows.values()]
    assert np.median(ratio) < 0.8 and all(r["profiled"]["evals"] > r["plain"]["evals"] for r in cmp_rows.values())
    # the networks on the same held-out seeds: Z = 1 agrees between the two runs (same solver)
    new = {e["seed"]: e for e in prof["eval"]}
    assert set(new) == set(cmp_rows)
    assert all(new[s]["z1"]["sweeps"] == cmp_rows[s]["z1"] for s in new)
    assert np.median([new[s]["learned"]["sweeps"] for s in new]) < 0.8 * np.median(
        [cmp_rows[s]["learned"] for s in new])


@pytest.mark.parametrize("dims,block,sigma", [((32, 32), (16, 16), 0.0), ((12, 11), (4, 5), 1.0),
                                               ((9, 8, 7), (4, 4, 3), 0.7)])
def test_line_pairs_match_oracle(vtmlib, dims, block, sigma):
    """Candidate couplings of §7.2: the same set of line pairs, with |a_ik|, as the oracle."""
    from oracle import coupled

    A = inputs.grid_poisson(dims, sigma=sigma, seed=4)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    pr, w = part.line_pairs()
    opr, ow = coupled.adjacent_line_pairs(evs.split_grid(A, dims, block), A)
    assert len(pr) == len(opr) > 0
    # line ids may be numbered differently; a line is identified by its two copies
    q, oq = part.lines(), evs.split_grid(A, dims, block).vtl
    got = {frozenset((tuple(q[t]), tuple(q[u]))): x for (t, u), x in zip(pr, w)}
    ref = {frozenset((tuple(int(v) for v in oq[t]), tuple(int(v) for v in oq[u]))): x for (t, u), x in zip(opr, ow)}
    assert got.keys() == ref.keys()
    assert all(got[k] == ref[k] for k in ref)
    assert np.all(pr[:, 0] < pr[:, 1])


@pytest.mark.parametrize("nx,ny,bx,by,rho,lam", [(12, 10, 2, 2, 0.6, 0.5), (16, 9, 4, 2, 0.9, 0.35),
                                                  (9, 9, 3, 1, 0.3, 0.7)])
def test_conformal_partition_matches_oracle(vtmlib, nx, ny, bx, by, rho, lam):
    """App. 1's general SPD split on a matrix that is not diagonally dominant: the library's
    (Cholesky-based) pieces, shares and lines against the oracle's (LU-based) to rounding."""
    from oracle import conformal
    from test_oracle_conformal import _block_home

    A = inputs.grid_anisotropic9(nx, ny, rho)
    home = _block_home(nx, ny, bx, by)
    with pytest.raises(vtmlib.VTMError):   # the diagonal rule cannot split it
        owners = [tuple(sorted({int(home[i])} | {int(home[k]) for k in A.col[A.rowptr[i]:A.rowptr[i + 1]]}))
                  for i in range(A.n)]
        vtmlib.partition_evs(A, "owners", owners=owners, lines=[(0, owners[0][0], owners[0][0])][:0])
    part = vtmlib.partition_evs(A, "conformal", home=home, lam=lam)
    _compare_split(part, conformal.split_conformal(A, home, lam=lam), atol=1e-13)
    assert part.info().nlines == len(conformal.split_conformal(A, home, lam=lam).vtl)


def test_conformal_partition_errors(vtmlib):
    A = inputs.grid_anisotropic9(6, 6, 0.5)
    home = np.zeros(A.n, np.int32)
    home[18:] = 1
    for kw in (dict(home=home, lam=0.0), dict(home=home, lam=1.0), dict(home=home, npieces=3),
               dict(home=np.full(A.n, 2, np.int32), npieces=2)):
        with pytest.raises(vtmlib.VTMError) as e:
            vtmlib.partition_evs(A, "conformal", **kw)
        assert e.value.code == 1
    # symmetric with a positive diagonal but indefinite: an interior Cholesky factor breaks down
    bad = inputs.csr_from_dense(np.eye(A.n) + 2.0 * (np.eye(A.n, k=1) + np.eye(A.n, k=-1)))
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.partition_evs(bad, "conformal", home=home)
    assert e.value.code == 4


def test_line_pairs_match_oracle_on_fem_split(vtmlib):
    """Candidate couplings on an unstructured split (RCB of element centroids, RCM local order):
    the same pairs of lines (identified by vertex and subgraphs) and weights as the oracle."""
    from oracle import coupled

    fem = inputs.fem_delaunay(3000, seed=14)
    part = vtmlib.partition_evs(fem.A, "elements", elements=dict(
        elem_nodes=fem.elem_nodes, elem_mats=fem.elem_mats, node_unknown=fem.node_unknown,
        elem_coords=fem.centroids), npieces=12)
    osplit = evs.split_by_elements(fem.A, fem.elem_nodes, fem.elem_mats, fem.node_unknown, evs.rcb(fem.centroids, 12))
    pr, w = part.line_pairs()
    opr, ow = coupled.adjacent_line_pairs(osplit, fem.A)
    q = part.lines()
    lib_key = [(int(part.piece(int(a))[0][la]), frozenset((int(a), int(b)))) for a, la, b, lb in q]
    or_key = [(int(osplit.subgraphs[a].vertices[la]), frozenset((int(a), int(b)))) for a, la, b, lb in osplit.vtl]
    got = {frozenset((lib_key[t], lib_key[u])): x for (t, u), x in zip(pr, w)}
    ref = {frozenset((or_key[t], or_key[u])): x for (t, u), x in zip(opr, ow)}
    assert len(got) == len(pr) > 0 and got.keys() == ref.keys()
    assert all(abs(got[k] - ref[k]) <= 1e-15 * abs(ref[k]) for k in ref)


def test_header_is_plain_c_and_links(vtmlib, tmp_path):
    """include/vtm.h is a C ABI: it compiles as C99 (-pedantic) and a C program links against the
    library and calls it (host-only entry points)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include "vtm.h"\n'
                   "int main(void) {\n"
                   "  vtm_setup_opts o = {0}; vtm_partition_spec sp = {0}; (void)o; (void)sp;\n"
                   "  int64_t out[2];\n"
                   "  double coords[4] = {0.0, 1.0, 2.0, 3.0};\n"
                   "  int32_t parts[4];\n"
                   "  if (vtm_rcb(coords, 4, 1, 2, parts) != VTM_OK) return 2;\n"
                   "  (void)out;\n"
                   "  return vtm_version() == 1 && parts[0] != parts[3] ? 0 : 1;\n"
                   "}\n")
    libdir = os.path.dirname(vtmlib.library_path())
    exe = tmp_path / "t"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lvtm", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0
