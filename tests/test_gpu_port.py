"""Port-response form of the sweep (u = u_base + S_j s with S_j = P^T K_j^{-1} P) against the oracle.

The form computes the same iterates as the band sweep (Table 1, eq. 5.6 / 5.8), so the tolerances
are those of the band path: 1e-12 (max norm, relative) in FP64 and TOL_FP32 in FP32 after k sweeps
(k - 1 port sweeps and one band sweep), residual 1e-10 (FP64) / 1e-8 (FP32 with defect
correction) at convergence.
"""
import numpy as np
import pytest

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from test_precision_bounds import TOL_FP16, TOL_FP32  # noqa: F401
from test_gpu_parity import _line_map, _oracle_after, _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", TOL_FP32)])
@pytest.mark.parametrize("nrhs", [1, 2, 8])
@pytest.mark.parametrize("dims,block", [((21, 19, 18), (8, 8, 8)), ((23, 17), (6, 5)), ((40, 33), (13, 11))])
def test_port_form_sweeps_match_oracle(vtmlib, precision, tol, nrhs, dims, block):
    """Grid splits with 2- and 3-cube corners (ports with 2 or 3 line ends), ragged last blocks,
    port counts that are not multiples of the 32-port tile (one to several tile rows)."""
    A = inputs.grid_poisson(dims, sigma=0.8, seed=21)
    b = inputs.rhs_uniform(A.n, nrhs, seed=21)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=0.7, precision=precision, nrhs=nrhs, form="port")
    assert s.info().sweep_form == 2 and s.info().port_bytes > 0
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    copies, waves = _oracle_after(osplit, b, 0.7, 7)
    assert _rel(s.copies(), copies) <= tol
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol
    # a further batch continues from the stored waves
    s.iterate(3)
    copies, waves = _oracle_after(osplit, b, 0.7, 10)
    assert _rel(s.copies(), copies) <= tol
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol


def test_port_form_random_owners_fp64(vtmlib):
    """Multilevel owner split of a random SPD matrix with per-line impedances (Thm 6.1 setting)."""
    A = inputs.random_dd_spd(400, avg_degree=5, excess=0.05, seed=3)
    As = A.to_scipy()
    rng = np.random.default_rng(3)
    home = rng.integers(0, 9, A.n)
    home[:9] = np.arange(9)
    owners = [tuple(sorted({int(home[i])} | {int(h) for h in home[As.indices[As.indptr[i]:As.indptr[i + 1]]]}))
              for i in range(A.n)]
    lines = [(i, p, q) for i, o in enumerate(owners) for a, p in enumerate(o) for q in o[a + 1:]]
    part = vtmlib.partition_evs(A, "owners", owners=owners, lines=lines)
    osplit = evs.split_by_owners(As, owners, lines)
    Z = np.exp(rng.uniform(np.log(0.2), np.log(5), len(lines)))
    b = inputs.rhs_uniform(A.n, 2, seed=3)
    s = vtmlib.Solver(part, z=Z, precision="fp64", nrhs=2, form="port")
    s.set_rhs(b)
    s.reset()
    s.iterate(6)
    copies, waves = _oracle_after(osplit, b, Z, 6)
    assert _rel(s.copies(), copies) <= 1e-12
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= 1e-12


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 1e-8)])
def test_port_form_solve(vtmlib, precision, rtol):
    dims, block = (33, 29, 17), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=22)
    b = inputs.rhs_uniform(A.n, 2, seed=22)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=1.0, precision=precision, nrhs=2, form="port")
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=rtol, maxit=20000)
    As = A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= rtol) and st.rel_residual <= rtol
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(x - xs)) <= 1e3 * rtol * np.max(np.abs(xs))
    # the same iteration as the band form: as many sweeps up to the check granularity, which the
    # port form stretches (batches sized from the observed rate, at most 8 check intervals)
    sb = vtmlib.Solver(part, z=1.0, precision=precision, nrhs=2, form="band")
    xb = np.zeros_like(b)
    stb = sb.solve(b, xb, rtol=rtol, maxit=20000)
    assert stb.sweeps - 20 <= st.sweeps <= 1.2 * stb.sweeps + 80


def test_port_form_auto_choice(vtmlib):
    """AUTO takes the port form where S_j is smaller than the band traffic of a batch (3D cubes) and
    where the tensor-core form applies (FP32, 16 / 32 right-hand sides); FP64 with 16 right-hand
    sides has no port form."""
    dims, block = (33, 33, 33), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=23)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    assert vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=1).info().sweep_form == 2
    assert vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=16).info().sweep_form == 2
    assert vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=16, form="band").info().sweep_form == 1
    dims2, block2 = (40, 33), (13, 11)
    A2 = inputs.grid_poisson(dims2, sigma=1.0, seed=23)
    part2 = vtmlib.partition_evs(A2, "grid", dims=dims2, block=block2)
    assert vtmlib.Solver(part2, z=1.0, precision="fp64", nrhs=16).info().sweep_form == 1
    with pytest.raises(vtmlib.VTMError):
        vtmlib.Solver(part2, z=1.0, precision="fp64", nrhs=16, form="port")


# Tensor-core form (R = 16 / 32): three TF32 products per term (hi(S) hi(s) + hi(S) lo(s) +
# lo(S) hi(s)) leave errors below 2^-21 of |S||s|, FP32 accumulation: the FP32 tolerance of the
# band path (TOL_FP32 = 6e-5 of the max norm after 7 sweeps) applies, which a single TF32 product
# exceeds about 30-fold (test_precision_bounds.py), and the solve with FP64 defect correction
# reaches 1e-8.
@pytest.mark.parametrize("nrhs", [16, 32])
@pytest.mark.parametrize("dims,block", [((21, 19, 18), (8, 8, 8)), ((34, 34, 34), (16, 16, 16)),
                                        ((40, 33), (13, 11))])
def test_port_tc_sweeps_match_oracle(vtmlib, nrhs, dims, block):
    """One to seven 128-port super-rows per subgraph (34^3 in 16^3 blocks: up to 817 ports), so the
    transposed products of the off-diagonal super-blocks and the zero padding are all exercised."""
    A = inputs.grid_poisson(dims, sigma=0.8, seed=24)
    b = inputs.rhs_uniform(A.n, nrhs, seed=24)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=0.7, precision="fp32", nrhs=nrhs, form="port")
    assert s.info().sweep_form == 2
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    copies, waves = _oracle_after(osplit, b, 0.7, 7)
    assert _rel(s.copies(), copies) <= TOL_FP32
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= TOL_FP32


@pytest.mark.parametrize("nrhs", [16, 32])
def test_port_tc_solve(vtmlib, nrhs):
    dims, block = (34, 30, 33), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=25)
    b = inputs.rhs_uniform(A.n, nrhs, seed=25)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=nrhs, form="port")
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=20000)
    As = A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= 1e-8) and st.rel_residual <= 1e-8
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(x - xs)) <= 1e-5 * np.max(np.abs(xs))


def _fem(vtmlib, npts, parts, seed):
    fem = inputs.fem_delaunay(npts, seed=seed)
    part = vtmlib.partition_evs(fem.A, "elements", elements=dict(elem_nodes=fem.elem_nodes, elem_mats=fem.elem_mats,
                                                               node_unknown=fem.node_unknown,
                                                               elem_coords=fem.centroids), npieces=parts)
    osplit = evs.split_by_elements(fem.A, fem.elem_nodes, fem.elem_mats, fem.node_unknown,
                                   evs.rcb(fem.centroids, parts))
    return fem, part, osplit


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", TOL_FP32)])
def test_port_form_fem_matches_oracle(vtmlib, precision, tol):
    """Uneven FEM subgraphs (RCB of element centroids, RCM order), stiffness-scaled impedances
    Z_t = 2 / (d_a + d_b): copies and waves after 7 sweeps against the oracle."""
    from test_gpu_fem import _maps
    fem, part, osplit = _fem(vtmlib, 5000, 20, seed=12)
    f = part.line_features()
    d = np.exp(f[:, 1].astype(np.float64))
    Z = 2.0 / (d[0::2] + d[1::2])
    b = inputs.rhs_uniform(fem.A.n, 2, seed=12)
    s = vtmlib.Solver(part, z=Z, precision=precision, nrhs=2, form="port")
    assert s.info().flagged_pieces == 0
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    cmap, emap = _maps(part, osplit)
    # oracle line order -> library line order for the impedances
    zl = np.empty(len(osplit.vtl))
    zl[emap[0::2] // 2] = Z
    m = ovtm.VTM(osplit, zl)
    st = m.initial_state(2)
    for _ in range(7):
        st = m.sweep(st, b)
    ref_c = np.concatenate([st.x_local[j] for j in range(len(osplit.subgraphs))], axis=1)
    assert _rel(s.copies(), ref_c[:, cmap]) <= tol
    assert _rel(s.get_state(), m.waves_out(st)[:, emap]) <= tol


def test_port_tc_fem_matches_oracle(vtmlib):
    """Uneven FEM subgraphs (one partial super-row each) with 16 right-hand sides on the tensor
    cores, stiffness-scaled impedances, 7 sweeps against the oracle."""
    from test_gpu_fem import _maps
    fem, part, osplit = _fem(vtmlib, 5000, 20, seed=13)
    f = part.line_features()
    d = np.exp(f[:, 1].astype(np.float64))
    Z = 2.0 / (d[0::2] + d[1::2])
    b = inputs.rhs_uniform(fem.A.n, 16, seed=13)
    s = vtmlib.Solver(part, z=Z, precision="fp32", nrhs=16, form="port")
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    cmap, emap = _maps(part, osplit)
    zl = np.empty(len(osplit.vtl))
    zl[emap[0::2] // 2] = Z
    m = ovtm.VTM(osplit, zl)
    st = m.initial_state(16)
    for _ in range(7):
        st = m.sweep(st, b)
    ref_c = np.concatenate([st.x_local[j] for j in range(len(osplit.subgraphs))], axis=1)
    assert _rel(s.copies(), ref_c[:, cmap]) <= TOL_FP32
    assert _rel(s.get_state(), m.waves_out(st)[:, emap]) <= TOL_FP32


def test_port_form_skips_flagged_subgraphs(vtmlib):
    """Z = 1e4 leaves some subgraphs nearly floating; their FP32 factorisations are flagged and they
    keep the FP64 band sweep in every sweep, so port responses are stored for the others only."""
    fem, part, osplit = _fem(vtmlib, 6000, 24, seed=9)
    s = vtmlib.Solver(part, z=1e4, precision="fp32", form="port")
    bits = s.piece_precision()
    assert s.info().flagged_pieces == int(np.sum(bits == 64)) >= 1
    la = part.lines()
    ports = [set() for _ in range(part.info().npieces)]
    for (pa, ca, pb, cb) in la:
        ports[int(pa)].add(int(ca))
        ports[int(pb)].add(int(cb))
    tiles = sum(((len(p) + 31) // 32) * ((len(p) + 31) // 32 + 1) // 2
                for j, p in enumerate(ports) if bits[j] == 32)
    assert s.info().port_bytes == tiles * 32 * 32 * 4
    b = inputs.rhs_uniform(fem.A.n, 1, seed=9)
    s.set_rhs(b)
    s.reset()
    s.iterate(5)
    assert np.isfinite(s.copies()).all() and np.isfinite(s.get_state()).all()


# FP16 storage of S_j (FP32 solvers): each 32 x 32 tile of S_j is divided by its largest entry and
# rounded to half (unit roundoff u16 = 2^-11 = 4.9e-4 of that entry); products stay FP32.  After 7
# sweeps the copies and waves stay within TOL_FP16 = 1e-3 (about 2 u16; observed up to 2.3e-4, the
# numpy emulation of test_precision_bounds.py 3.6e-4) and the FP32 bound TOL_FP32 would see the
# FP16 rounding.  The solve with FP64 defect correction must still reach 1e-8.
@pytest.mark.parametrize("nrhs", [1, 2])
@pytest.mark.parametrize("dims,block", [((21, 19, 18), (8, 8, 8)), ((40, 33), (13, 11))])
def test_port_fp16_sweeps_match_oracle(vtmlib, nrhs, dims, block):
    A = inputs.grid_poisson(dims, sigma=0.8, seed=26)
    b = inputs.rhs_uniform(A.n, nrhs, seed=26)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=0.7, precision="fp32", nrhs=nrhs, form="port", port_storage="fp16")
    assert s.info().port_storage_bits == 16
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    copies, waves = _oracle_after(osplit, b, 0.7, 7)
    assert _rel(s.copies(), copies) <= TOL_FP16
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= TOL_FP16


@pytest.mark.parametrize("storage", ["fp16", "fp16-auto"])
def test_port_fp16_solve(vtmlib, storage):
    dims, block = (33, 29, 17), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=27)
    b = inputs.rhs_uniform(A.n, 2, seed=27)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=2, form="port", port_storage=storage)
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=20000)
    As = A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= 1e-8)
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(x - xs)) <= 1e-5 * np.max(np.abs(xs))


def test_port_fp16_auto_on_high_contrast_fem(vtmlib):
    """The 1e-3/1e3 FEM checkerboard converges slowly; FP16_AUTO must still reach 1e-8."""
    fem, part, osplit = _fem(vtmlib, 4000, 16, seed=6)
    f = part.line_features()
    d = np.exp(f[:, 1].astype(np.float64))
    Z = 6.0 / (d[0::2] + d[1::2])
    b = inputs.rhs_uniform(fem.A.n, 2, seed=6)
    s = vtmlib.Solver(part, z=Z, precision="fp32", nrhs=2, form="port", port_storage="fp16-auto")
    x = np.zeros_like(b)
    s.solve(b, x, rtol=1e-8, maxit=100000)
    As = fem.A.to_scipy()
    rel = np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    assert np.all(rel <= 1e-8)
    assert s.info().port_storage_bits in (16, 32)


@pytest.mark.parametrize("coupling", [None, 1.0])
def test_port_fp16_auto_large_responses(vtmlib, coupling):
    """Responses larger than 96 MB (64^3, 0.19 GB FP32): FP16_AUTO takes the FP16 copy, for coupled
    lines with the FP16-floor restart rule; the solve reaches 1e-8 both ways, twice in a row."""
    dims, block = (64, 64, 64), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=28)
    b = inputs.rhs_uniform(A.n, 1, seed=28)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=4.0 if coupling else 1.0, precision="fp32", form="port", port_storage="fp16-auto",
                      coupling=coupling, check_every=20)
    assert s.info().port_storage_bits == 16
    As = A.to_scipy()
    for _ in range(2):
        x = np.zeros_like(b)
        s.solve(b, x, rtol=1e-8, maxit=20000)
        assert np.linalg.norm(b[0] - As @ x[0]) / np.linalg.norm(b[0]) <= 1e-8
