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


def _csr_dev(A):
    return (torch.tensor(A.rowptr, device="cuda"), torch.tensor(A.col, device="cuda"),
            torch.tensor(A.val, device="cuda"))


def test_noalloc_eight_rhs_strided_and_zero_column(vtmlib):
    """The nrhs limit (8), leading dimensions larger than n through the C ABI, and a zero column of
    b (rel = ||A x_r|| there), against the host residual, twice in a row."""
    import ctypes as C
    A = inputs.grid_poisson((24, 20), sigma=0.8, seed=4)
    n, R, ld = A.n, 8, A.n + 37
    rng = np.random.default_rng(4)
    b = rng.uniform(-1, 1, (R, n))
    b[3] = 0.0
    x = rng.uniform(-1, 1, (R, n))
    As = A.to_scipy()
    res = np.linalg.norm(b - (As @ x.T).T, axis=1)
    nb = np.linalg.norm(b, axis=1)
    expect = np.where(nb > 0, res / np.where(nb > 0, nb, 1), res)
    bpad = torch.full((R, ld), float("nan"), dtype=torch.float64, device="cuda")
    xpad = torch.full((R, ld), float("nan"), dtype=torch.float64, device="cuda")
    bpad[:, :n] = torch.tensor(b, device="cuda")
    xpad[:, :n] = torch.tensor(x, device="cuda")
    rowptr, col, val = _csr_dev(A)
    rel = torch.empty(R, dtype=torch.float64, device="cuda")
    lib = vtmlib._lib
    for _ in range(2):
        rel.fill_(float("nan"))
        code = lib.vtm_relative_residual_noalloc(n, C.c_void_p(rowptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                                 C.c_void_p(val.data_ptr()), R, C.c_void_p(bpad.data_ptr()), ld,
                                                 C.c_void_p(xpad.data_ptr()), ld, C.c_void_p(rel.data_ptr()), None)
        assert code == 0, lib.vtm_last_error()
        torch.cuda.synchronize()
        assert np.allclose(rel.cpu().numpy(), expect, rtol=1e-12, atol=0)


def test_noalloc_allocates_nothing_on_repeated_calls(vtmlib):
    """After a first call on the device, further calls leave the device's free memory unchanged."""
    A = inputs.grid_poisson((40, 40), sigma=0.5, seed=6)
    rowptr, col, val = _csr_dev(A)
    b = torch.tensor(inputs.rhs_uniform(A.n, 4, seed=6), device="cuda")
    x = torch.zeros_like(b)
    rel = torch.empty(4, dtype=torch.float64, device="cuda")
    vtmlib.relative_residual_noalloc(rowptr, col, val, b, x, rel)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        vtmlib.relative_residual_noalloc(rowptr, col, val, b, x, rel)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.allclose(rel.cpu().numpy(), 1.0)     # x = 0: ||b|| / ||b||


def test_noalloc_binding_rejects_bad_arguments(vtmlib):
    A = inputs.grid_poisson((8, 8))
    rowptr, col, val = _csr_dev(A)
    b = torch.ones((2, A.n), dtype=torch.float64, device="cuda")
    rel = torch.empty(2, dtype=torch.float64, device="cuda")
    bad = [dict(x=torch.ones((2, A.n + 1), dtype=torch.float64, device="cuda")),   # x larger than b
           dict(rel=torch.empty(1, dtype=torch.float64, device="cuda")),          # rel too short
           dict(x=torch.ones((A.n, 2), dtype=torch.float64, device="cuda").t()),  # not contiguous
           dict(col=col.to(torch.int64)),                                          # wrong index type
           dict(x=torch.ones((2, A.n), dtype=torch.float32, device="cuda")),      # wrong value type
           dict(x=torch.ones((2, A.n), dtype=torch.float64))]                     # host tensor
    for kw in bad:
        args = dict(rowptr=rowptr, col=col, val=val, b=b, x=b, rel=rel)
        args.update(kw)
        with pytest.raises(ValueError):
            vtmlib.relative_residual_noalloc(**args)
