"""The allocation-free residual entry point against the solver's own residual (GPU).

vtm_relative_residual_noalloc exists for callers that cannot allocate device memory when they call
it (a process whose device memory is reserved up front by a caching allocator, or a loop that must
not let cudaMalloc/cudaFree synchronise the device).  Its only scratch is a fixed 128-byte device
array inside the library.  This file is collected last on purpose so that a stop-at-first-failure
run has already run every other test; it must also pass alone in a fresh process.
"""
import numpy as np
import pytest

from paper_0807_1949_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_noalloc_residual_matches_solve_twice(vtmlib):
    A = inputs.grid_poisson((32, 32), sigma=0.5, seed=2)
    b = inputs.rhs_uniform(A.n, 2, seed=2)
    part = vtmlib.partition_evs(A, "grid", dims=(32, 32), block=(16, 16))
    s = vtmlib.Solver(part, z=1.0, precision="fp64", nrhs=2)
    bd = torch.tensor(b, device="cuda")
    xd = torch.zeros_like(bd)
    st = s.solve(bd, xd, rtol=1e-10, maxit=5000)
    assert st.rel_residual <= 1e-10
    rowptr = torch.tensor(A.rowptr, device="cuda")
    col = torch.tensor(A.col, device="cuda")
    val = torch.tensor(A.val, device="cuda")
    rel = torch.empty(2, dtype=torch.float64, device="cuda")
    x = xd.cpu().numpy()
    expect_rhs = np.linalg.norm(b - (A.to_scipy() @ x.T).T, axis=1) / np.linalg.norm(b, axis=1)
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        rel.fill_(float("nan"))
        vtmlib.relative_residual_noalloc(rowptr, col, val, bd, xd, rel)
        torch.cuda.synchronize()
        got = rel.cpu().numpy()
        assert abs(got.max() - st.rel_residual) <= 1e-12 * st.rel_residual
        assert np.allclose(got, expect_rhs, rtol=1e-10, atol=0)


def test_noalloc_rejects_too_many_rhs(vtmlib):
    n = 4
    rowptr = torch.arange(0, n + 1, dtype=torch.int64, device="cuda")
    col = torch.arange(0, n, dtype=torch.int32, device="cuda")
    val = torch.ones(n, dtype=torch.float64, device="cuda")
    b = torch.ones((9, n), dtype=torch.float64, device="cuda")
    rel = torch.empty(9, dtype=torch.float64, device="cuda")
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.relative_residual_noalloc(rowptr, col, val, b, b, rel)
    assert e.value.code == 1 and "nrhs" in str(e.value)
