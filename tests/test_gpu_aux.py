"""Auxiliary subsystems on the device: the residual history of a solve (metrics) and run-to-run
reproducibility of the sweeps (the race check: a kernel that races shows as bit differences
between identical runs)."""
import numpy as np
import pytest

from paper_0807_1949_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 1e-8)])
def test_solve_history(vtmlib, precision, rtol):
    dims, block = (33, 29, 17), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=1.0, seed=51)
    b = inputs.rhs_uniform(A.n, 2, seed=51)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=2.0, precision=precision, nrhs=2, coupling=0.5, check_every=10)
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=rtol, maxit=20000)
    sw, rel, inner = s.history()
    assert len(sw) == st.checks >= 2
    assert np.all(np.diff(sw) > 0) and sw[-1] == st.sweeps
    assert rel[-1] == st.rel_residual and rel[-1] <= rtol and np.all(rel[:-1] > rtol)
    assert inner[0] == rel[0]
    As = A.to_scipy()
    assert np.max(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)) == pytest.approx(rel[-1], rel=1e-6)


@pytest.mark.parametrize("precision,nrhs", [("fp64", 1), ("fp32", 2), ("fp32", 16), ("fp64", 16)])
def test_band_sweeps_are_bitwise_reproducible(vtmlib, precision, nrhs):
    """Band sweeps reduce in a fixed order (warp shuffles, no atomics): identical runs agree bit for
    bit, coupled lines included."""
    dims, block = (40, 37, 21), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=0.9, seed=52)
    b = inputs.rhs_uniform(A.n, nrhs, seed=52)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    out = []
    for _ in range(2):
        s = vtmlib.Solver(part, z=2.0, precision=precision, nrhs=nrhs, form="band", coupling=0.5)
        s.set_rhs(b)
        s.reset()
        s.iterate(12)
        out.append((s.get_state(), s.copies()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("precision,nrhs,storage", [("fp64", 1, "native"), ("fp32", 1, "fp16"), ("fp32", 2, "native"),
                                                    ("fp32", 16, "native"), ("fp32", 32, "fp16")])
def test_port_sweeps_are_bitwise_reproducible(vtmlib, precision, nrhs, storage):
    """The SIMT port sweep hands each block row of S_j to one warp and sums the warps' column parts in
    a fixed order; the tensor-core sweep issues its products from one thread in a fixed order and
    reduces its column maxima without atomics.  Identical runs agree bit for bit, coupled lines
    included."""
    dims, block = (40, 37, 21), (8, 8, 8)
    A = inputs.grid_poisson(dims, sigma=0.9, seed=53)
    b = inputs.rhs_uniform(A.n, nrhs, seed=53)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    out = []
    for _ in range(2):
        s = vtmlib.Solver(part, z=2.0, precision=precision, nrhs=nrhs, form="port", coupling=0.5, port_storage=storage)
        assert s.info().sweep_form == 2
        s.set_rhs(b)
        s.reset()
        s.iterate(12)
        out.append((s.get_state(), s.copies()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
