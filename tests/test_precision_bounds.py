"""The parity tolerances of the reduced-precision GPU paths, and why they can tell the schemes apart.

The GPU parity tests compare copies and waves after k sweeps with the FP64 oracle in the max norm,
relative to the largest entry.  Their bounds (``TOL_FP32``, ``TOL_FP16``) are set a little above
the largest error observed on a GB300 and are derived from the arithmetic:

* FP32 factors and sweeps, and the tensor-core port sweep with three TF32 products per term
  (hi(S) hi(s) + hi(S) lo(s) + lo(S) hi(s)): the FP32 banded Cholesky has backward error of order
  (w + 1) u32 (|L||L^T|), w the half-bandwidth, u32 = 2^-24; on 17^3 subgraphs (w = 289) that is
  1.7e-5, and the three-product split leaves below 2^-21 of |S||s| per term.  Observed maximum
  over every FP32 / 3xTF32 parity case: 2.9e-5 (34^3 in 16^3 blocks, 32 right-hand sides, after
  10 sweeps); 2.4e-5 for the benchmarked configuration with FP32 storage.  ``TOL_FP32`` = 6e-5
  (about 2^10 u32).
* FP16 storage of the port responses: each 32 x 32 tile of S_j is scaled by its largest entry and
  rounded to half, unit roundoff u16 = 2^-11 = 4.9e-4 of that entry; the products stay FP32.
  Observed maximum 2.9e-4 (the benchmarked configuration after 10 sweeps); the numpy emulation
  below reaches 3.6e-4 on the FP16 parity case.  ``TOL_FP16`` = 1e-3 (about 2 u16).

A single TF32 product per term (unit roundoff 2^-11, the operands truncated to 10 mantissa bits)
must fail ``TOL_FP32``, or the tensor-core tests could not see a lost split.  The test below runs
the port form of the same sweeps in numpy with the products emulated both ways (everything else in
FP64) and checks that the one-product scheme exceeds the bound several times over while the
three-product scheme stays far below it.
"""
import numpy as np
import pytest

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs

TOL_FP32 = 6e-5
TOL_FP16 = 1e-3


def tf32(x):
    """Truncate FP32 values to TF32 (sign, 8 exponent bits, 10 mantissa bits), as the tensor core
    reads a 32-bit operand."""
    b = np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def product(S, s, scheme):
    """S @ s with the tensor core's operand rounding: 'tf32x1' = hi(S) hi(s); 'tf32x3' adds
    hi(S) lo(s) + lo(S) hi(s) with lo = x - hi(x) (exact in FP32, read as TF32); FP64 accumulation
    (the tensor core accumulates in FP32, far below these terms)."""
    S32, s32 = np.asarray(S, np.float32), np.asarray(s, np.float32)
    hS, hs = tf32(S32), tf32(s32)
    if scheme == "tf32x1":
        return hS @ hs
    lS = tf32(S32.astype(np.float64) - hS)
    ls = tf32(s32.astype(np.float64) - hs)
    return hS @ hs + hS @ ls + lS @ hs


class PortForm:
    """The port-response form of the sweep in FP64 (u = u_base + S_j s, S_j = P^T K_j^{-1} P), from
    the oracle's local matrices; only the product S_j s is emulated."""

    def __init__(self, split, Z, b):
        self.m = ovtm.VTM(split, Z)
        e = self.m.ends
        self.ends = e
        self.ports, self.S, self.ubase, self.end_port = [], [], [], np.empty(len(e.piece), np.int64)
        b = np.atleast_2d(b)
        off = 0
        for j, g in enumerate(split.subgraphs):
            mine = np.nonzero(e.piece == j)[0]
            ports = np.unique(e.local[mine])
            pos = {int(c): k for k, c in enumerate(ports)}
            for t in mine:
                self.end_port[t] = off + pos[int(e.local[t])]
            off += len(ports)
            n = len(g.vertices)
            unit = np.zeros((len(ports), n))
            unit[np.arange(len(ports)), ports] = 1.0
            Kinv_P = self.m.factor[j].solve(unit)                  # (nports, n): rows K^{-1} e_c
            self.S.append(Kinv_P[:, ports])
            self.ubase.append(self.m.factor[j].solve(split.local_rhs(b, j))[:, ports].T)
            self.ports.append(ports)
        self.R = b.shape[0]

    def sweep(self, w_out_prev, scheme, S_list=None):
        e = self.ends
        S_list = self.S if S_list is None else S_list
        w_in = w_out_prev[:, e.twin]                               # (R, E)
        nports = len(self.end_port) and int(self.end_port.max()) + 1
        s = np.zeros((nports, self.R))
        np.add.at(s, self.end_port, (w_in / e.Z[None, :]).T)
        u = np.empty_like(s)
        off = 0
        for j, S in enumerate(S_list):
            k = len(self.ports[j])
            sj = s[off:off + k]
            y = S @ sj if scheme == "fp64" else product(S, sj, scheme)
            u[off:off + k] = self.ubase[j] + y
            off += k
        return 2.0 * u[self.end_port].T - w_in


@pytest.mark.parametrize("dims,block,nrhs", [((21, 19, 18), (8, 8, 8), 16), ((40, 33), (13, 11), 32)])
def test_single_tf32_product_fails_the_fp32_bound(dims, block, nrhs):
    """The tensor-core parity cases (same grids, seed, Z = 0.7): six port sweeps then one exact
    sweep, as vtm_iterate(7) runs them.  One TF32 product exceeds TOL_FP32 at least 3x; three stay
    below TOL_FP32 / 5; FP64 products reproduce the oracle (checks the emulation itself)."""
    A = inputs.grid_poisson(dims, sigma=0.8, seed=24)
    b = inputs.rhs_uniform(A.n, nrhs, seed=24)
    split = evs.split_grid(A, dims, block)
    pf = PortForm(split, 0.7, b)
    m = pf.m
    st = m.initial_state(nrhs)
    for _ in range(7):
        st = m.sweep(st, b)
    ref = m.waves_out(st)
    err = {}
    for scheme in ("fp64", "tf32x1", "tf32x3"):
        w = np.zeros((nrhs, len(pf.ends.piece)))
        for _ in range(6):
            w = pf.sweep(w, scheme)
        w = pf.sweep(w, "fp64")
        err[scheme] = np.max(np.abs(w - ref)) / np.max(np.abs(ref))
    assert err["fp64"] <= 1e-12
    assert err["tf32x1"] >= 3 * TOL_FP32, err
    assert err["tf32x3"] <= TOL_FP32 / 5, err


def test_fp16_tile_rounding_stays_inside_its_bound():
    """FP16 storage emulated on the FP16 parity case (21 x 19 x 18 in 8^3 blocks, Z = 0.7): every
    32 x 32 tile of S_j divided by its largest entry and rounded to half, products in FP64; after
    seven sweeps (six port sweeps, one exact) the waves stay within TOL_FP16 and above TOL_FP32
    (FP16 storage is visible to the FP32 bound)."""
    dims, block, nrhs = (21, 19, 18), (8, 8, 8), 2
    A = inputs.grid_poisson(dims, sigma=0.8, seed=26)
    b = inputs.rhs_uniform(A.n, nrhs, seed=26)
    split = evs.split_grid(A, dims, block)
    pf = PortForm(split, 0.7, b)
    half = []
    for S in pf.S:
        k = S.shape[0]
        Sh = np.empty_like(S)
        for I in range(0, k, 32):
            for J in range(0, k, 32):
                t = S[I:I + 32, J:J + 32]
                sc = np.max(np.abs(t)) or 1.0
                Sh[I:I + 32, J:J + 32] = (t / sc).astype(np.float16).astype(np.float64) * sc
        half.append(Sh)
    st = pf.m.initial_state(nrhs)
    for _ in range(7):
        st = pf.m.sweep(st, b)
    ref = pf.m.waves_out(st)
    w = np.zeros((nrhs, len(pf.ends.piece)))
    for _ in range(6):
        w = pf.sweep(w, "fp64", half)
    w = pf.sweep(w, "fp64")
    err = np.max(np.abs(w - ref)) / np.max(np.abs(ref))
    assert TOL_FP32 < err <= TOL_FP16 / 2, err
