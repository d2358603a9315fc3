"""Mixed-precision VTM with FP64 defect correction — oracle for error statements.  TEST
INFRASTRUCTURE ONLY.

The iteration of Table 1 is run with the local factors of eq. 5.8 stored in a reduced precision
(FP32, BF16 or FP16) and the local solves carried out in that precision (FP32 arithmetic for FP32
storage; the narrower formats are widened to FP32 for the arithmetic, as a kernel would), while the
residual b - A x, the accumulated solution and the convergence test stay in FP64.  The outer loop
is classical defect correction (iterative refinement): the sweeps solve A d = r from zero boundary
variables, x <- x + d, r <- b - A x in FP64, and the sweeps restart on the new r once the inner
residual has dropped by ``inner_reduction`` or stalls.  This is the structure the library's FP32
solve uses; the FP64 oracle (vtm.py) remains the reference for every result.

Why the outer loop is needed: inexact local solves are exact solves of perturbed local matrices,
i.e. a different split of a perturbed A, so the inner iteration converges to the solution of a
perturbed system.  Its error relative to the true correction is set by the storage precision, the
local condition numbers and, through the slow modes, by how close the iteration's spectral radius
is to 1.  Each outer step gains that many digits.

Precisions (unit roundoff u): fp32 2^-24, bf16 2^-8, fp16 2^-11 (range 6e-5 .. 65504 for normals).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .evs import SplitGraph, _as_csr
from .vtm import VTM


def round_to(a: np.ndarray, kind: str) -> np.ndarray:
    """Values of ``a`` rounded to the storage format ``kind`` (round to nearest even), as float64."""
    if kind == "fp64":
        return np.asarray(a, dtype=np.float64)
    if kind == "fp32":
        return np.asarray(a, dtype=np.float32).astype(np.float64)
    if kind == "fp16":
        return np.asarray(a, dtype=np.float16).astype(np.float64)
    if kind == "bf16":
        x = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        u = x.view(np.uint32).astype(np.uint64)
        # nearest even on the 16 bits that are dropped
        r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
        return (r << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(kind)


class MixedVTM(VTM):
    """Table 1 with the banded Cholesky factor of every K_j rounded to ``kind`` and the substitution
    done in FP32 arithmetic (FP64 for kind = "fp64")."""

    def __init__(self, split: SplitGraph, Z, kind: str = "fp32"):
        super().__init__(split, Z)
        self.kind = kind
        dt = np.float64 if kind == "fp64" else np.float32
        for f in self.factor.values():
            f.cb = round_to(f.cb, kind).astype(dt)
        self._dt = dt

    def local_solve(self, j: int, r: np.ndarray) -> np.ndarray:
        f = self.factor[j]
        return sla.cho_solve_banded((f.cb, True), np.asarray(r, dtype=self._dt).T).T.astype(np.float64)

    def sweep(self, state, b, pieces=None):
        # the FP64 sweep of VTM with the local solve replaced: same right-hand side (eq. 5.8) and
        # current update; the right-hand side is rounded to the working precision by local_solve
        saved = {j: self.factor[j].solve for j in self.pieces}
        try:
            for j in self.pieces:
                self.factor[j].solve = (lambda r, j=j: self.local_solve(j, r))
            return super().sweep(state, b, pieces)
        finally:
            for j in self.pieces:
                self.factor[j].solve = saved[j]


@dataclass
class RefinedResult:
    x: np.ndarray
    sweeps: int
    restarts: int
    history: list = field(default_factory=list)   # (sweeps, max relative residual) at every check


def solve_refined(split: SplitGraph, A, b: np.ndarray, Z, kind: str = "fp32", rtol: float = 1e-8,
                  maxit: int = 10000, check_every: int = 10, inner_reduction: float = 1e-4) -> RefinedResult:
    """FP64 defect correction around reduced-precision VTM sweeps (module docstring)."""
    m = MixedVTM(split, Z, kind)
    As = _as_csr(A)
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    x = np.zeros_like(b)
    r = b.copy()
    rn = np.linalg.norm(r, axis=1)
    sweeps = restarts = 0
    hist = []
    xt = x
    while sweeps < maxit:
        st = m.initial_state(b.shape[0])
        inner_sweeps = 0
        prev = np.inf
        restarted = False
        while sweeps < maxit:
            for _ in range(min(check_every, maxit - sweeps)):
                st = m.sweep(st, r)
                sweeps += 1
                inner_sweeps += 1
            xt = x + m.assemble(st)
            rt = b - (As @ xt.T).T
            rel = np.linalg.norm(rt, axis=1) / np.linalg.norm(b, axis=1)
            inner = float(np.max(np.linalg.norm(rt, axis=1) / rn))
            hist.append((sweeps, float(np.max(rel))))
            if np.max(rel) <= rtol:
                return RefinedResult(x=xt, sweeps=sweeps, restarts=restarts, history=hist)
            if inner < 1.0 and (inner <= inner_reduction or (inner >= 0.98 * prev and inner_sweeps >= 2 * check_every)):
                x, r = xt, rt
                rn = np.maximum(np.linalg.norm(r, axis=1), 1e-300)
                restarts += 1
                restarted = True
                break
            prev = inner
        if not restarted:
            break
    return RefinedResult(x=xt, sweeps=sweeps, restarts=restarts, history=hist)
