"""Failure detection and checkpoint/resume through the C ABI (GPU).

No test faults, traps or hangs the GPU: the timeout test withholds one bulk copy so that the
bounded mbarrier wait can only run out; the kernel then records VTM_ERR_TIMEOUT, drains the copies
it did issue and returns, and the context stays usable.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_0807_1949_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _grid(vtmlib, dims=(40, 36), block=(16, 12), sigma=0.5):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=1)
    return A, vtmlib.partition_evs(A, "grid", dims=dims, block=block)


@pytest.mark.parametrize("precision,nrhs", [("fp64", 1), ("fp32", 16)])
def test_bounded_wait_reports_timeout_and_context_survives(vtmlib, precision, nrhs):
    A, part = _grid(vtmlib)
    b = inputs.rhs_uniform(A.n, nrhs, seed=1)
    s = vtmlib.Solver(part, z=1.0, precision=precision, nrhs=nrhs, wait_polls=256, withhold_slab=2)
    x = np.zeros_like(b)
    with pytest.raises(vtmlib.VTMError) as e:
        s.solve(b, x, rtol=1e-8, maxit=100)
    assert e.value.code == 7
    del s
    ok = vtmlib.Solver(part, z=1.0, precision=precision, nrhs=nrhs)
    st = ok.solve(b, x, rtol=1e-8, maxit=20000)
    assert st.rel_residual <= 1e-8


def test_not_converged_and_diverged(vtmlib):
    A, part = _grid(vtmlib)
    b = inputs.rhs_uniform(A.n, 1, seed=2)
    s = vtmlib.Solver(part, z=1.0, precision="fp64")
    x = np.zeros_like(b)
    st = s.solve(b, x, rtol=1e-12, maxit=20, raise_on_fail=False)
    assert st.status == 5 and st.sweeps == 20 and np.all(np.isfinite(x))
    bad = b.copy()
    bad[0, 7] = np.nan
    st = s.solve(bad, x, rtol=1e-8, maxit=100, raise_on_fail=False)
    assert st.status == 6


def test_not_spd_local_matrix(vtmlib):
    """A non-conformal explicit split (an indefinite piece) fails the factorisation (Cor. 4.1)."""
    A = inputs.csr_from_dense(np.array([[4.0, -1.0, 0.0], [-1.0, 4.0, -1.0], [0.0, -1.0, 4.0]]))
    P1 = sp.csr_matrix(np.array([[4.0, -1.0], [-1.0, -2.0]]))   # vertex 1's share made negative
    P2 = sp.csr_matrix(np.array([[6.0, -1.0], [-1.0, 4.0]]))
    blk = sp.block_diag([P1, P2]).tocsr()
    cols = blk.indices.copy()
    cols[blk.indptr[2]:] -= 2
    spec = dict(piece_ptr=[0, 2, 4], copy_vertex=[0, 1, 1, 2], copy_share=[1.0, 0.5, 0.5, 1.0],
                local_rowptr=blk.indptr, local_col=cols, local_val=blk.data, line_copy_a=[1], line_copy_b=[2])
    part = vtmlib.partition_evs(A, "explicit", explicit=spec)
    with pytest.raises(vtmlib.VTMError) as e:
        vtmlib.Solver(part, z=100.0, precision="fp64")
    assert e.value.code == 4


@pytest.mark.parametrize("precision,nrhs", [("fp64", 1), ("fp32", 2), ("fp32", 16)])
def test_checkpoint_resume_is_bitwise(vtmlib, precision, nrhs):
    """Table 1's whole state is the waves: stopping after 3 sweeps and resuming from the saved
    waves in a new solver reproduces 7 uninterrupted sweeps bit for bit."""
    A, part = _grid(vtmlib)
    b = inputs.rhs_uniform(A.n, nrhs, seed=3)
    s1 = vtmlib.Solver(part, z=0.9, precision=precision, nrhs=nrhs)
    s1.set_rhs(b)
    s1.reset()
    s1.iterate(3)
    saved = s1.get_state()
    s1.iterate(4)
    ref_w, ref_x = s1.get_state(), s1.copies()
    s2 = vtmlib.Solver(part, z=0.9, precision=precision, nrhs=nrhs)
    s2.set_rhs(b)
    s2.reset()
    s2.set_state(saved)
    s2.iterate(4)
    assert np.array_equal(s2.get_state(), ref_w)
    assert np.array_equal(s2.copies(), ref_x)
