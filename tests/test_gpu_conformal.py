"""The solver on App. 1's general conformal split (VTM_PART_CONFORMAL) of SPD matrices that are not
diagonally dominant: sweeps against the FP64 oracle iterating the oracle's own split (pieces equal
to rounding, tests/test_host.py), and solves to tolerance.  Tolerances as in the other parity
tests: 1e-12 in FP64 and TOL_FP32 (6e-5) in FP32 after k sweeps."""
import numpy as np
import pytest

from oracle import conformal
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs
from test_precision_bounds import TOL_FP16, TOL_FP32  # noqa: F401
from test_gpu_parity import _line_map, _oracle_after, _rel
from test_oracle_conformal import _block_home

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", TOL_FP32)])
@pytest.mark.parametrize("nrhs,form", [(1, "band"), (2, "port"), (16, "band")])
def test_conformal_sweeps_match_oracle(vtmlib, precision, tol, nrhs, form):
    nx, ny = 30, 22
    A = inputs.grid_anisotropic9(nx, ny, 0.7)
    home = _block_home(nx, ny, 4, 2)
    part = vtmlib.partition_evs(A, "conformal", home=home, lam=0.4)
    osplit = conformal.split_conformal(A, home, lam=0.4)
    b = inputs.rhs_uniform(A.n, nrhs, seed=41)
    s = vtmlib.Solver(part, z=1.5, precision=precision, nrhs=nrhs, form=form)
    s.set_rhs(b)
    s.reset()
    s.iterate(8)
    copies, waves = _oracle_after(osplit, b, 1.5, 8)
    assert _rel(s.copies(), copies) <= tol
    assert _rel(s.get_state(), waves[:, _line_map(part, osplit)]) <= tol


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-10), ("fp32", 1e-8)])
def test_conformal_solve(vtmlib, precision, rtol):
    """Thm 6.1 on SPD pieces: the solve reaches the tolerance and the direct solution."""
    nx, ny = 48, 40
    A = inputs.grid_anisotropic9(nx, ny, 0.8)
    part = vtmlib.partition_evs(A, "conformal", home=_block_home(nx, ny, 4, 4))
    b = inputs.rhs_uniform(A.n, 2, seed=42)
    s = vtmlib.Solver(part, z=1.0, precision=precision, nrhs=2)
    x = np.zeros_like(b)
    s.solve(b, x, rtol=rtol, maxit=20000)
    As = A.to_scipy()
    assert np.all(np.linalg.norm(b - (As @ x.T).T, axis=1) / np.linalg.norm(b, axis=1) <= rtol)
    xs = ovtm.direct_solve(As, b)
    assert np.max(np.abs(x - xs)) <= 1e3 * rtol * np.max(np.abs(xs))
