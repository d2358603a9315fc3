"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: FP64 path 1e-12 relative (max norm) on copies and waves after k sweeps, relative
residual <= 1e-10 at convergence; FP32 path: the sweep-level tolerance TOL_FP32 = 6e-5 of the max
norm comes from the FP32 band Cholesky's backward error (~(w+1) u_32 |L||L^T|; its derivation and
the observed errors are in test_precision_bounds.py), and the defect-corrected solve must reach
relative residual <= 1e-8.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from test_precision_bounds import TOL_FP16, TOL_FP32  # noqa: F401
from conftest import load_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _line_map(part, osplit):
    """Index of each library line end (2t+side) in the oracle's end order."""
    idx = {tuple(int(x) for x in q): t for t, q in enumerate(osplit.vtl)}
    out = []
    for q in part.lines():
        t = idx[tuple(int(x) for x in q)]
        out += [2 * t, 2 * t + 1]
    return np.array(out)


def _oracle_after(osplit, b, Z, k):
    m = ovtm.VTM(osplit, Z)
    st = m.initial_state(np.atleast_2d(b).shape[0])
    for _ in range(k):
        st = m.sweep(st, b)
    copies = np.concatenate([st.x_local[j] for j in range(len(osplit.subgraphs))], axis=1)
    return copies, m.waves_out(st)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("k", [1, 2, 7, 30])
def test_config1_fp64_sweeps_match_oracle(vtmlib, k):
    """2D Laplacian 32x32, 4 pieces, Z = 1, FP64: copies and waves after k sweeps."""
    A = inputs.grid_poisson((32, 32))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    part = vtmlib.partition_evs(A, "grid", dims=(32, 32), block=(16, 16))
    osplit = evs.split_grid(A, (32, 32), (16, 16))
    s = vtmlib.Solver(part, z=1.0, precision="fp64")
    s.set_rhs(b)
    s.reset()
    s.iterate(k)
    copies, waves = _oracle_after(osplit, b, 1.0, k)
    assert _rel(s.copies(), copies) <= 1e-12
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= 1e-12


def test_config1_fp64_solve_to_1e10(vtmlib):
    A = inputs.grid_poisson((32, 32))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    part = vtmlib.partition_evs(A, "grid", dims=(32, 32), block=(16, 16))
    s = vtmlib.Solver(part, z=1.0, precision="fp64", check_every=2)
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-10, maxit=5000)
    r = np.linalg.norm(b[0] - A.to_scipy() @ x[0]) / np.linalg.norm(b[0])
    assert r <= 1e-10 and st.rel_residual <= 1e-10
    osol = ovtm.solve(evs.split_grid(A, (32, 32), (16, 16)), A, b, 1.0, rtol=1e-10, maxit=5000)
    assert osol.sweeps <= st.sweeps <= osol.sweeps + 2
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(x - xs)) <= 1e-8 * np.max(np.abs(xs))
    # device pointers through torch
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    s.solve(bt, xt, rtol=1e-10, maxit=5000)
    assert np.max(np.abs(xt.cpu().numpy() - x)) <= 1e-14 * np.max(np.abs(x))


def test_example_5_1_fp64(vtmlib):
    """Example 5.1 (explicit split of eq. 4.1/4.2, Z3 = 1, Z4 = 0.5) for 20 sweeps from zero."""
    from test_host import example_explicit
    from test_oracle import example_split
    A, b, spec = example_explicit(load_golden)
    part = vtmlib.partition_evs(A, "explicit", explicit=spec)
    osplit = example_split()
    Z = np.array(load_golden("example_5_1.json")["Z"])
    s = vtmlib.Solver(part, z=Z, precision="fp64")
    s.set_rhs(b[None, :])
    s.reset()
    s.iterate(20)
    copies, waves = _oracle_after(osplit, b, Z, 20)
    assert _rel(s.copies(), copies) <= 1e-12
    assert _rel(s.get_state(), waves) <= 1e-12
    x = np.zeros((1, 6))
    s.solve(b[None, :], x, rtol=1e-13, maxit=400)
    assert np.allclose(x[0], np.linalg.solve(A.to_dense(), b), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_random_multilevel_fp64(vtmlib, seed):
    """Random SPD, multilevel owner split, random per-line Z (Thm 6.1 setting), nrhs = 2."""
    A = inputs.random_dd_spd(300, avg_degree=4, excess=0.05, seed=seed)
    As = A.to_scipy()
    rng = np.random.default_rng(seed)
    home = rng.integers(0, 7, A.n)
    home[:7] = np.arange(7)
    owners = [tuple(sorted({int(home[i])} | {int(h) for h in home[As.indices[As.indptr[i]:As.indptr[i + 1]]]}))
              for i in range(A.n)]
    lines = [(i, p, q) for i, o in enumerate(owners) for a, p in enumerate(o) for q in o[a + 1:]]
    part = vtmlib.partition_evs(A, "owners", owners=owners, lines=lines)
    osplit = evs.split_by_owners(As, owners, lines)
    Z = np.exp(rng.uniform(np.log(0.1), np.log(10), len(lines)))
    # library line order equals the given line order for the owners kind
    b = inputs.rhs_uniform(A.n, 2, seed=seed)
    s = vtmlib.Solver(part, z=Z, precision="fp64", nrhs=2)
    s.set_rhs(b)
    s.reset()
    s.iterate(5)
    copies, waves = _oracle_after(osplit, b, Z, 5)
    assert _rel(s.copies(), copies) <= 1e-12
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= 1e-12
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-10, maxit=20000)
    assert np.all(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1) <= 1e-10)


@pytest.mark.parametrize("nrhs", [1, 4, 16, 32])
def test_3d_fp32_sweeps_and_refined_solve(vtmlib, nrhs):
    """3D variable-coefficient grid (ragged blocks), FP32 factors: sweeps within the FP32 bound,
    defect-corrected solve to 1e-8 and the direct solution."""
    dims, block = (21, 19, 18), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=4)
    b = inputs.rhs_uniform(A.n, nrhs, seed=4)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=nrhs, form="band")
    s.set_rhs(b)
    s.reset()
    s.iterate(3)
    copies, waves = _oracle_after(osplit, b, 1.0, 3)
    assert _rel(s.copies(), copies) <= TOL_FP32
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= TOL_FP32
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=20000)
    As = A.to_scipy()
    assert np.all(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1) <= 1e-8)
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(x - xs)) <= 1e-6 * np.max(np.abs(xs))


@pytest.mark.parametrize("variant", ["single", "pipelined"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", TOL_FP32)])
@pytest.mark.parametrize("nrhs", [1, 2])
@pytest.mark.parametrize("dims,block", [((21, 19, 18), (8, 8, 8)), ((23, 17), (6, 5)), ((70, 9), (70, 9))])
def test_sweep_variants_match_oracle(vtmlib, variant, precision, tol, nrhs, dims, block):
    """Both substitution schedules of the sweep (one block step at a time; chain warp plus
    look-ahead warps) against the oracle after 5 sweeps: ragged 3D blocks (several 32-row blocks per
    subgraph), 2D blocks of 30 unknowns (one block: the forward/backward turn is the only step) and
    one subgraph of half-bandwidth 70 (20 blocks, a non-empty far part in every row, no lines)."""
    A = inputs.grid_poisson(dims, sigma=0.7, seed=11)
    b = inputs.rhs_uniform(A.n, nrhs, seed=11)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=0.9, precision=precision, nrhs=nrhs, sweep_variant=variant)
    assert s.info().sweep_variant == (1 if variant == "pipelined" else 0)
    s.set_rhs(b)
    s.reset()
    s.iterate(5)
    copies, waves = _oracle_after(osplit, b, 0.9, 5)
    assert _rel(s.copies(), copies) <= tol
    if len(osplit.vtl):
        assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol


def test_pipelined_variant_needs_nrhs_le_2(vtmlib):
    A = inputs.grid_poisson((16, 16))
    part = vtmlib.partition_evs(A, "grid", dims=(16, 16), block=(8, 8))
    with pytest.raises(vtmlib.VTMError):
        vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=4, sweep_variant="pipelined")


def test_wide_fp64_matches_oracle(vtmlib):
    """The windowed multi-RHS kernel in FP64 (16 right-hand sides) against the oracle, 4 sweeps."""
    dims, block = (23, 17), (8, 6)
    A = inputs.grid_poisson(dims, sigma=1.2, seed=8)
    b = inputs.rhs_uniform(A.n, 16, seed=8)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=0.8, precision="fp64", nrhs=16)
    s.set_rhs(b)
    s.reset()
    s.iterate(4)
    copies, waves = _oracle_after(osplit, b, 0.8, 4)
    assert _rel(s.copies(), copies) <= 1e-12
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= 1e-12


def test_config2_full_size_sampled(vtmlib):
    """128^3, sigma = 1, 512 pieces, FP32 (the benchmarked launch): sweep 1 from zero waves on
    sampled pieces against the oracle's banded solve of those pieces, then the refined solve."""
    dims, block = (128, 128, 128), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=0)
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    info = part.info()
    assert info.npieces == 512
    s = vtmlib.Solver(part, z=1.0, precision="fp32")
    s.set_rhs(b)
    s.reset()
    s.iterate(1)
    xc = s.copies()[0]
    offs = np.concatenate([[0], np.cumsum([part.piece(j)[0].size for j in range(512)])])
    for j in (0, 7, 73, 292, 511):
        v, Aj, share = evs.split_grid_piece(A, dims, block, j)
        ports = evs.grid_piece_line_count(dims, block, j)
        K = (Aj + sp.diags(ports.astype(float) / 1.0)).tocsr()
        ref = ovtm.BandedCholesky(K).solve((b[:, v] * share))[0]
        got = xc[offs[j]:offs[j + 1]]
        assert _rel(got, ref) <= TOL_FP32, (j, _rel(got, ref))
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=20000)
    r = np.linalg.norm(b[0] - A.to_scipy() @ x[0]) / np.linalg.norm(b[0])
    assert r <= 1e-8, (r, st.sweeps)


@pytest.mark.parametrize("dims,block,sigma", [((32, 32), (16, 16), 0.0), ((21, 19, 18), (8, 8, 8), 1.0)])
def test_fp32_solve_matches_mixed_oracle(vtmlib, dims, block, sigma):
    """The library's FP32 sweeps inside FP64 defect correction against the mixed-precision oracle
    (factors rounded to FP32, FP32 substitution, the same restart rule): both reach 1e-8 with about
    the same sweeps and restarts; the factors differ only in rounding (the GPU factors in FP32)."""
    from oracle import mixed
    A = inputs.grid_poisson(dims, sigma=sigma, seed=3)
    b = inputs.rhs_uniform(A.n, 1, seed=3)
    osplit = evs.split_grid(A, dims, block)
    ref = mixed.solve_refined(osplit, A, b, 1.0, kind="fp32", rtol=1e-8, maxit=20000, check_every=10)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", check_every=10, form="band")
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-8, maxit=20000)
    assert ref.history[-1][1] <= 1e-8 and st.rel_residual <= 1e-8
    assert abs(st.sweeps - ref.sweeps) <= max(20, 0.1 * ref.sweeps)
    assert abs(st.restarts - ref.restarts) <= 1
