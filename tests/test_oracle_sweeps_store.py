"""The stored sweep counts of the plain method (tests/golden/oracle_sweeps.json, written by
tests/golden/make_oracle_sweeps.py from the oracle alone) against a live rerun of the oracle: the
32^2 entry whole, the 256^2 entry's residuals at its first two stored checks.  The benchmark's
reference arm takes its sweep counts from this file."""
import numpy as np

from conftest import load_golden
from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def _problem(dims, block, sigma):
    A = inputs.grid_poisson(dims, sigma=sigma, seed=0)
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    return A, b, evs.split_grid(A, dims, block)


def test_stored_32x32_count_is_the_oracles():
    g = load_golden("oracle_sweeps.json")["laplace2d-32"]
    A, b, split = _problem((32, 32), (16, 16), 0.0)
    res = ovtm.solve(split, A, b, 1.0, rtol=1e-8, maxit=100000, check_every=10)
    assert res.sweeps == g["sweeps"] == 150
    assert np.isclose(res.history[-1][1], g["rel_residual"], rtol=1e-9)


def test_stored_256x256_history_is_the_oracles():
    """Residuals after 10 and 110 sweeps (Z = 1, zero initial waves) as stored; the count itself
    (4010, the plain FP64 method's count on the GPU as well) took about six minutes on one core."""
    g = load_golden("oracle_sweeps.json")["poisson2d-256"]
    assert g["sweeps"] == 4010 and g["rel_residual"] <= 1e-8
    A, b, split = _problem((256, 256), (32, 32), 1.25)
    res = ovtm.solve(split, A, b, 1.0, rtol=1e-30, maxit=110, check_every=10)
    got = dict(res.history)
    for k, r in g["history"][:2]:
        assert k in (10, 110) and np.isclose(got[k], r, rtol=1e-9), (k, got[k], r)
