"""Coupled virtual transmission lines (§7.2, Thm 7.1) on the device against the coupled oracle.

The bundle admittance is Y = diag(1/Z_t) + sum_p y_p (e_t - e_t')(e_t - e_t')^T over the candidate
pairs of Partition.line_pairs() with y_p = gamma |a_ik|.  The coupled sweep computes the same
iterates as oracle/coupled.py, so the tolerances are those of the uncoupled paths: 1e-12 (max
norm, relative) in FP64 and TOL_FP32 (6e-5) in FP32 after k sweeps, in both sweep forms.
"""
import numpy as np
import pytest

from oracle import coupled, evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from test_precision_bounds import TOL_FP16, TOL_FP32  # noqa: F401
from test_gpu_parity import _line_map, _rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _problem(vtmlib, dims, block, sigma, seed, z, gamma):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=seed)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    pr, w = part.line_pairs()
    idx = {tuple(int(x) for x in q): t for t, q in enumerate(osplit.vtl)}
    lib_to_or = np.array([idx[tuple(int(x) for x in q)] for q in part.lines()])
    zl = np.broadcast_to(np.asarray(z, dtype=np.float64), (len(lib_to_or),))
    zo = np.empty_like(zl)
    zo[lib_to_or] = zl
    y = gamma * w
    Y = coupled.laplacian_admittance(osplit, zo, lib_to_or[pr], y)
    return A, part, osplit, (pr, y), Y


def _oracle_after(osplit, Y, b, k):
    m = coupled.CoupledVTM(osplit, Y)
    st = m.initial_state(np.atleast_2d(b).shape[0])
    for _ in range(k):
        st = m.sweep(st, b)
    copies = np.concatenate([st.x_local[j] for j in range(len(osplit.subgraphs))], axis=1)
    return copies, m.waves_out(st)


CASES = [("fp64", 1e-12, 1, "band"), ("fp64", 1e-12, 2, "port"), ("fp64", 1e-12, 8, "port"),
         ("fp64", 1e-12, 16, "band"), ("fp32", TOL_FP32, 1, "band"), ("fp32", TOL_FP32, 1, "port"),
         ("fp32", TOL_FP32, 8, "port"), ("fp32", TOL_FP32, 16, "port"), ("fp32", TOL_FP32, 32, "port"),
         ("fp32", TOL_FP32, 32, "band")]


@pytest.mark.parametrize("precision,tol,nrhs,form", CASES)
@pytest.mark.parametrize("dims,block", [((21, 19, 18), (8, 8, 8)), ((40, 33), (13, 11))])
def test_coupled_sweeps_match_oracle(vtmlib, precision, tol, nrhs, form, dims, block):
    """Ragged grid splits with 2- and 3-cube corners; per-line impedances; 7 then 10 sweeps."""
    nl = vtmlib.partition_evs(inputs.grid_poisson(dims), "grid", dims=dims, block=block).info().nlines
    z = np.random.default_rng(2).uniform(1.0, 4.0, nl)
    A, part, osplit, cpl, Y = _problem(vtmlib, dims, block, 0.8, 21, z, 0.5)
    b = inputs.rhs_uniform(A.n, nrhs, seed=21)
    s = vtmlib.Solver(part, z=z, precision=precision, nrhs=nrhs, form=form, coupling=cpl)
    assert s.info().ncouplings == len(cpl[1]) > 0
    assert s.info().sweep_form == (2 if form == "port" else 1)
    s.set_rhs(b)
    s.reset()
    s.iterate(7)
    copies, waves = _oracle_after(osplit, Y, b, 7)
    assert _rel(s.copies(), copies) <= tol
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol
    s.iterate(3)
    copies, waves = _oracle_after(osplit, Y, b, 10)
    assert _rel(s.copies(), copies) <= tol
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol


def test_zero_conductances_are_the_uncoupled_method(vtmlib):
    dims, block = (23, 17), (6, 5)
    A = inputs.grid_poisson(dims, sigma=0.5, seed=3)
    b = inputs.rhs_uniform(A.n, 2, seed=3)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    pr, w = part.line_pairs()
    s0 = vtmlib.Solver(part, z=1.3, nrhs=2)
    s1 = vtmlib.Solver(part, z=1.3, nrhs=2, coupling=(pr, 0 * w))
    assert s1.info().ncouplings == 0
    for s in (s0, s1):
        s.set_rhs(b)
        s.reset()
        s.iterate(5)
    assert np.array_equal(s0.get_state(), s1.get_state())


@pytest.mark.parametrize("precision,form,rtol", [("fp64", "band", 1e-10), ("fp32", "port", 1e-8),
                                                 ("fp32", "band", 1e-8)])
def test_coupled_solve_converges_and_beats_uncoupled(vtmlib, precision, form, rtol):
    """Thm 7.1 on the device, and the effect that motivates the coupling: with the tangential
    conductance the larger Z that damps the smooth interface modes no longer slows the rough
    ones, so the solve needs far fewer sweeps than the best uniform uncoupled Z of a small scan."""
    dims, block = (32, 32, 32), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=1)
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    As = A.to_scipy()
    x = np.zeros_like(b)
    s = vtmlib.Solver(part, z=4.0, precision=precision, nrhs=1, form=form, coupling=0.5, check_every=5)
    st = s.solve(b, x, rtol=rtol, maxit=5000)
    assert np.linalg.norm(b - (As @ x.T).T) / np.linalg.norm(b) <= rtol
    xs = ovtm.direct_solve(As, b)
    assert np.max(np.abs(x - xs)) <= 1e3 * rtol * np.max(np.abs(xs))
    best = 10 ** 9
    for z in (0.5, 1.0, 2.0, 4.0):
        x0 = np.zeros_like(b)
        best = min(best, vtmlib.Solver(part, z=z, precision=precision, nrhs=1, form=form,
                                       check_every=5).solve(b, x0, rtol=rtol, maxit=5000).sweeps)
    assert st.sweeps < 0.6 * best


def test_coupled_matched_and_learned_modes(vtmlib):
    """MATCHED impedances are computed on the uncoupled lines, then the couplings are added."""
    dims, block = (24, 20, 16), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=0.7, seed=5)
    b = inputs.rhs_uniform(A.n, 1, seed=5)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z="matched", coupling=0.25)
    x = np.zeros_like(b)
    s.solve(b, x, rtol=1e-10, maxit=5000)
    As = A.to_scipy()
    assert np.linalg.norm(b - (As @ x.T).T) / np.linalg.norm(b) <= 1e-10


def test_invalid_couplings_are_rejected(vtmlib):
    dims, block = (20, 20), (7, 7)
    A = inputs.grid_poisson(dims)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    pr, w = part.line_pairs()
    q = part.lines()
    bundle = [frozenset((a[0], a[2])) for a in q]
    t0 = int(pr[0, 0])
    other = next(u for u in range(len(q)) if bundle[u] != bundle[t0])
    far = next(u for u in range(len(q)) if bundle[u] == bundle[t0] and u != t0 and
               not any((min(t0, u), max(t0, u)) == (int(a), int(c)) for a, c in pr))
    bad = [([[t0, other]], [1.0]), ([[t0, far]], [1.0]), ([[t0, t0]], [1.0]), ([[t0, len(q)]], [1.0]),
           ([pr[0]], [-1.0]), ([pr[0]], [np.nan])]
    for pairs, y in bad:
        with pytest.raises(vtmlib.VTMError) as e:
            vtmlib.Solver(part, z=1.0, coupling=(np.array(pairs), np.array(y)))
        assert e.value.code == 1  # VTM_ERR_INVALID
    s = vtmlib.Solver(part, z=1.0, coupling=0.5)
    with pytest.raises(vtmlib.VTMError) as e:
        s.input_impedances()
    assert e.value.code == 1  # VTM_ERR_INVALID


def _fem_coupled(vtmlib, npts, parts, seed, zscale, gamma):
    from test_gpu_fem import _maps
    from test_gpu_port import _fem
    fem, part, osplit = _fem(vtmlib, npts, parts, seed)
    cmap, emap = _maps(part, osplit)
    f = part.line_features()
    d = np.exp(f[:, 1].astype(np.float64))
    Z = zscale / (d[0::2] + d[1::2])
    lib_to_or = emap[0::2] // 2
    zo = np.empty(len(osplit.vtl))
    zo[lib_to_or] = Z
    pr, w = part.line_pairs()
    Y = coupled.laplacian_admittance(osplit, zo, lib_to_or[pr], gamma * w)
    return fem, part, osplit, cmap, emap, Z, (pr, gamma * w), Y


@pytest.mark.parametrize("nrhs,form", [(1, "band"), (2, "port"), (16, "band")])
def test_coupled_fem_fp64_matches_oracle(vtmlib, nrhs, form):
    """Unstructured split (RCB of FEM element centroids, RCM local order): candidate pairs from
    the library's partition, coupled sweeps against the coupled oracle."""
    fem, part, osplit, cmap, emap, Z, cpl, Y = _fem_coupled(vtmlib, 4000, 16, 31, 8.0, 1.0)
    assert len(cpl[1]) > 0
    b = inputs.rhs_uniform(fem.A.n, nrhs, seed=31)
    s = vtmlib.Solver(part, z=Z, precision="fp64", nrhs=nrhs, form=form, coupling=cpl)
    s.set_rhs(b)
    s.reset()
    s.iterate(6)
    copies, waves = _oracle_after(osplit, Y, b, 6)
    assert _rel(s.copies(), copies[:, cmap]) <= 1e-12
    assert _rel(s.get_state(), waves[:, emap]) <= 1e-12


def test_coupled_fem_fp32_solve(vtmlib):
    """The 1e-3/1e3 checkerboard FEM with coupled lines in FP32 port form reaches 1e-8."""
    fem, part, osplit, cmap, emap, Z, cpl, Y = _fem_coupled(vtmlib, 4000, 16, 6, 6.0, 1.0)
    b = inputs.rhs_uniform(fem.A.n, 2, seed=6)
    s = vtmlib.Solver(part, z=Z, precision="fp32", nrhs=2, form="port", coupling=cpl)
    x = np.zeros_like(b)
    s.solve(b, x, rtol=1e-8, maxit=100000)
    As = fem.A.to_scipy()
    assert np.all(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1) <= 1e-8)


def test_coupled_with_flagged_subgraphs(vtmlib):
    """Z = 1e4 leaves subgraphs nearly floating; their FP32 factorisations are flagged and swept in
    FP64, with the coupling currents of their ports, beside the FP32 ones."""
    from test_gpu_port import _fem
    fem, part, osplit = _fem(vtmlib, 6000, 24, seed=9)
    s = vtmlib.Solver(part, z=1e4, precision="fp32", form="band", coupling=0.5)
    assert s.info().flagged_pieces >= 1 and s.info().ncouplings > 0
    b = inputs.rhs_uniform(fem.A.n, 1, seed=9)
    s.set_rhs(b)
    s.reset()
    s.iterate(5)
    assert np.isfinite(s.copies()).all() and np.isfinite(s.get_state()).all()
