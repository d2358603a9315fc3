"""Pins of the mixed-precision oracle (oracle/mixed.py): storage rounding, reduction to the FP64
oracle, the accuracy floor of reduced-precision sweeps without correction, and convergence of the
defect correction to the FP64 tolerance."""
import numpy as np
import pytest

from oracle import evs, mixed
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def test_round_to_formats():
    """Round to nearest, ties to even, in each format's own precision."""
    one = 1.0
    assert mixed.round_to(np.array([one / 3]), "fp32")[0] == float(np.float32(one / 3))
    # bf16 (7 stored mantissa bits): below half an ulp rounds down, a tie goes to the even mantissa
    assert mixed.round_to(np.array([1 + 2.0 ** -9]), "bf16")[0] == 1.0
    assert mixed.round_to(np.array([1 + 3 * 2.0 ** -8]), "bf16")[0] == 1 + 2.0 ** -6
    assert mixed.round_to(np.array([1 + 2.0 ** -8]), "bf16")[0] == 1.0
    # fp16 (10 stored bits): a tie at 1 + 2^-11 goes to 1
    assert mixed.round_to(np.array([1 + 2.0 ** -11]), "fp16")[0] == 1.0
    assert mixed.round_to(np.array([1 + 3 * 2.0 ** -11]), "fp16")[0] == 1 + 2.0 ** -9
    # relative error bound u = 2^-8 for bf16 on random values
    x = np.random.default_rng(0).uniform(-10, 10, 1000)
    assert np.max(np.abs(mixed.round_to(x, "bf16") - x) / np.abs(x)) <= 2.0 ** -8


def _laplace():
    A = inputs.grid_poisson((32, 32))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    return A, b, evs.split_grid(A, (32, 32), (16, 16))


def test_fp64_kind_is_the_oracle():
    """With FP64 storage the mixed iteration is the FP64 oracle's iteration."""
    A, b, sp = _laplace()
    m64, m = ovtm.VTM(sp, 1.0), mixed.MixedVTM(sp, 1.0, "fp64")
    s64, s = m64.initial_state(), m.initial_state()
    for _ in range(7):
        s64, s = m64.sweep(s64, b), m.sweep(s, b)
    assert np.array_equal(m64.waves_out(s64), m.waves_out(s))


def test_reduced_precision_floor_needs_correction():
    """Without the outer FP64 loop the sweeps stall at a floor set by the storage precision: FP32
    between the FP64 tolerance (1e-10) and 1e-5, BF16 far above it."""
    A, b, sp = _laplace()
    floors = {}
    for kind in ("fp32", "bf16"):
        m = mixed.MixedVTM(sp, 1.0, kind)
        st = m.initial_state()
        for _ in range(600):
            st = m.sweep(st, b)
        floors[kind] = float(ovtm.relative_residual(A, b, m.assemble(st))[0])
    assert 1e-10 < floors["fp32"] < 1e-5
    assert floors["bf16"] > 1e-4


@pytest.mark.parametrize("kind,max_restarts", [("fp32", 2), ("fp16", 6), ("bf16", 10)])
def test_defect_correction_reaches_fp64_tolerance(kind, max_restarts):
    """FP64 defect correction takes reduced-precision sweeps to 1e-8; the solution matches the
    direct solve to 1e-6 of its size.  Narrower storage costs restarts (error statement: FP32 needs
    the same sweeps as FP64 on this problem)."""
    A, b, sp = _laplace()
    r = mixed.solve_refined(sp, A, b, 1.0, kind=kind, rtol=1e-8, maxit=4000)
    assert r.history[-1][1] <= 1e-8
    assert 1 <= r.restarts <= max_restarts
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(r.x - xs)) <= 1e-6 * np.max(np.abs(xs))
    if kind == "fp32":
        o = ovtm.solve(sp, A, b, 1.0, rtol=1e-8, maxit=4000, check_every=10)
        assert abs(r.sweeps - o.sweeps) <= 10
