"""The multi-RHS band sweep with its products on the tensor cores (FP32, 16 / 32 right-hand sides)
against the FP64 oracle and against the same sweep without them (GPU).

Shapes cover one, two and three 128-column tiles left of a 128-row group (half-bandwidths 64 ..
324), ragged last groups and subgraphs of different sizes in one launch.
"""
import numpy as np
import pytest

from oracle import evs
from paper_0807_1949_gb300 import inputs
from test_gpu_parity import _line_map, _oracle_after, _rel
from test_precision_bounds import TOL_FP32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = [((21, 19, 18), (8, 8, 8), 1.0),       # w = 64: one tile, groups of 512 / 576 rows
         ((30, 25, 26), (12, 12, 12), 1.0),    # w = 144: two tiles, ragged groups
         ((34, 34, 34), (16, 16, 16), 1.5)]    # w up to 324: three tiles (the benchmarked shape)


@pytest.mark.parametrize("nrhs", [16, 32])
@pytest.mark.parametrize("dims,block,sigma", CASES)
def test_tensor_core_band_sweep_matches_oracle_and_simt(vtmlib, nrhs, dims, block, sigma):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=5)
    b = inputs.rhs_uniform(A.n, nrhs, seed=5)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    osplit = evs.split_grid(A, dims, block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=nrhs, form="band")
    assert s.info().band_tc == 1 and s.info().band_tc_bytes > 0
    s.set_rhs(b)
    s.reset()
    s.iterate(4)
    copies, waves = _oracle_after(osplit, b, 1.0, 4)
    assert _rel(s.copies(), copies) <= TOL_FP32
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= TOL_FP32
    simt = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=nrhs, form="band", sweep_variant="simt")
    assert simt.info().band_tc == 0
    simt.set_rhs(b)
    simt.reset()
    simt.iterate(4)
    assert _rel(s.copies(), simt.copies()) <= TOL_FP32


@pytest.mark.parametrize("nrhs", [16, 32])
def test_tensor_core_band_sweep_solves_to_1e8(vtmlib, nrhs):
    dims, block = (34, 34, 34), (16, 16, 16)
    A = inputs.grid_poisson(dims, sigma=1.5, seed=6)
    b = inputs.rhs_uniform(A.n, nrhs, seed=6)
    part = vtmlib.partition_evs(A, "grid", dims=dims, block=block)
    s = vtmlib.Solver(part, z=1.0, precision="fp32", nrhs=nrhs, form="band", check_every=20)
    assert s.info().band_tc == 1
    x = np.zeros_like(b)
    s.solve(b, x, rtol=1e-8, maxit=20000)
    As = A.to_scipy()
    assert np.all(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1) <= 1e-8)
