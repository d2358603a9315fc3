"""Virtual Transmission Method (paper §5, Table 1) — FP64 oracle.  TEST INFRASTRUCTURE ONLY.

Notation follows §5.  Every VTL end e sits at a port (local unknown c(e) of subgraph j(e)) and has
a twin end twin(e) on the other side of the same line; Z_e is the line's characteristic
impedance, equal at both ends.  Each end carries the paper's pair (u_e, omega_e): the port
potential and the inflow current through that line.  A port with several lines (multilevel EVS,
Fig. 7) has one potential and one current per line.

One iteration k (Table 1 steps 3-5, all subgraphs in parallel, synchronous):

* eq. 5.6 / 5.8, right-hand side:
      r_j = b̃_j + sum_e Z_e^{-1} (u_{twin(e)}^{k-1} - Z_e omega_{twin(e)}^{k-1}) at c(e)
* eq. 5.8, local SPD system with the lines' admittances on the port diagonal:
      K_j = Ã_j + sum_e Z_e^{-1} e_{c(e)} e_{c(e)}^T,   K_j x_j^k = r_j
  K_j is fixed, so it is factored once and every iteration is a forward/back substitution (§8).
  The factorisation is a library banded Cholesky (LAPACK pbtrf/pbtrs through scipy), the
  paper's "Sparse or Dense Cholesky" (§5).
* eq. 5.8, current update:
      u_e^k = x_j^k[c(e)],  omega_e^k = Z_e^{-1}(u_{twin(e)}^{k-1} - u_e^k) - omega_{twin(e)}^{k-1}
* Table 1 step 2: the initial pair is u^0 = omega^0 = 0 unless given.

Assembly (a reading: the paper only states the fixed point, where all copies agree, Thm 4.1):
x_i = mean of the copies of vertex i.  Convergence is measured as the FP64 relative residual
||b - A x||_2 / ||b||_2 per right-hand side; the paper's RMS error against the exact solution
(§7.1, §9) is available as ``rms_error``.

Pins: Example 5.1's local matrices (eq. 5.4/5.5) exactly; convergence of Example 5.1 to the
direct solution of eq. 3.2; the port-space operator of eq. A3.8 reproduces successive errors
(theory.py); single-line reflection closed form (theory.py); Thm 6.1 on random SPD splits;
Thm 4.1 at the fixed point (twins equal, currents opposite).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .evs import SplitGraph, _as_csr


@dataclass
class Ends:
    """VTL ends: end 2t is side a of line t, end 2t+1 side b; twin(2t) = 2t+1."""

    piece: np.ndarray   # j(e)
    local: np.ndarray   # c(e)
    twin: np.ndarray    # twin(e)
    Z: np.ndarray       # Z_e


def ends_of(split: SplitGraph, Z) -> Ends:
    m = len(split.vtl)
    Zl = np.broadcast_to(np.asarray(Z, dtype=np.float64), (m,)).copy()
    piece = np.empty(2 * m, dtype=np.int64)
    local = np.empty(2 * m, dtype=np.int64)
    piece[0::2], local[0::2] = split.vtl[:, 0], split.vtl[:, 1]
    piece[1::2], local[1::2] = split.vtl[:, 2], split.vtl[:, 3]
    twin = np.arange(2 * m) ^ 1
    return Ends(piece=piece, local=local, twin=twin, Z=np.repeat(Zl, 2))


def local_matrix(split: SplitGraph, ends: Ends, j: int) -> sp.csr_matrix:
    """K_j = Ã_j + sum over ends e at subgraph j of Z_e^{-1} e_c e_c^T (eq. 5.8)."""
    A = split.subgraphs[j].A.tolil(copy=True)
    for e in np.nonzero(ends.piece == j)[0]:
        c = ends.local[e]
        A[c, c] = A[c, c] + 1.0 / ends.Z[e]
    return A.tocsr()


class BandedCholesky:
    """Library banded Cholesky factor of a sparse SPD matrix (LAPACK pbtrf), solved by pbtrs."""

    def __init__(self, K: sp.spmatrix):
        K = sp.coo_matrix(K)
        n = K.shape[0]
        low = K.row >= K.col
        w = int(np.max(K.row[low] - K.col[low])) if n else 0
        ab = np.zeros((w + 1, n))
        ab[K.row[low] - K.col[low], K.col[low]] = K.data[low]
        self.n, self.w = n, w
        self.cb = sla.cholesky_banded(ab, lower=True)

    def solve(self, r: np.ndarray) -> np.ndarray:
        """r of shape (R, n) -> x of shape (R, n)."""
        return sla.cho_solve_banded((self.cb, True), np.asarray(r).T).T


@dataclass
class State:
    """The boundary variables of every end (Table 1) and the last local solutions."""

    u: np.ndarray      # (R, E)
    omega: np.ndarray  # (R, E)
    x_local: list      # per subgraph: (R, n_j) last local solution (None before sweep 1)


class VTM:
    """The method of Table 1 on a split graph with line impedances Z (scalar or per line)."""

    def __init__(self, split: SplitGraph, Z, pieces=None):
        self.split = split
        self.ends = ends_of(split, Z)
        self.pieces = range(len(split.subgraphs)) if pieces is None else list(pieces)
        self.factor = {j: BandedCholesky(local_matrix(split, self.ends, j)) for j in self.pieces}
        self.ends_at = {j: np.nonzero(self.ends.piece == j)[0] for j in range(len(split.subgraphs))}

    def initial_state(self, nrhs: int = 1) -> State:
        E = len(self.ends.piece)
        return State(u=np.zeros((nrhs, E)), omega=np.zeros((nrhs, E)), x_local=[None] * len(self.split.subgraphs))

    def sweep(self, state: State, b: np.ndarray, pieces=None) -> State:
        """One synchronous VTM iteration (Table 1 steps 3-5) over ``pieces`` (default all)."""
        b = np.atleast_2d(b)
        new_u = state.u.copy()
        new_om = state.omega.copy()
        x_local = list(state.x_local)
        todo = self.pieces if pieces is None else pieces
        for j in todo:
            x_local[j] = self.piece_step(j, state.u, state.omega, b, new_u, new_om)
        return State(u=new_u, omega=new_om, x_local=x_local)

    def piece_step(self, j: int, u: np.ndarray, omega: np.ndarray, b: np.ndarray, new_u: np.ndarray,
                   new_om: np.ndarray) -> np.ndarray:
        """Table 1 steps 3-5 for subgraph j: reads the twins' pair (u, omega) of the previous
        iteration from ``u``, ``omega`` and writes its own ends' new pair into ``new_u``,
        ``new_om``; returns the local solution (R, n_j)."""
        e = self.ends
        r = self.split.local_rhs(b, j).copy()
        mine = self.ends_at[j]
        for t in mine:                           # eq. 5.8 right-hand side, from eq. 5.6
            tw = e.twin[t]
            r[:, e.local[t]] += (u[:, tw] - e.Z[t] * omega[:, tw]) / e.Z[t]
        x = self.factor[j].solve(r)              # eq. 5.8 local SPD solve
        for t in mine:                           # current update after eq. 5.8
            tw = e.twin[t]
            new_u[:, t] = x[:, e.local[t]]
            new_om[:, t] = (u[:, tw] - new_u[:, t]) / e.Z[t] - omega[:, tw]
        return x

    def waves_out(self, state: State) -> np.ndarray:
        """Outgoing wave u_e - Z_e omega_e of each end: the left side of eq. 5.6 seen from the twin."""
        return state.u - self.ends.Z[None, :] * state.omega

    def assemble(self, state: State) -> np.ndarray:
        """x_i = mean over the copies of vertex i of the last local solutions; (R, n)."""
        return assemble(self.split, state)


def assemble(split: SplitGraph, state: State) -> np.ndarray:
    """x_i = mean over the copies of vertex i of the last local solutions; (R, n)."""
    R = state.u.shape[0]
    acc = np.zeros((R, split.n))
    cnt = np.zeros(split.n)
    for j, g in enumerate(split.subgraphs):
        if state.x_local[j] is None:
            continue
        np.add.at(acc.T, g.vertices, state.x_local[j].T)
        np.add.at(cnt, g.vertices, 1.0)
    return acc / np.maximum(cnt, 1.0)[None, :]


def relative_residual(A, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """||b - A x||_2 / ||b||_2 per right-hand side (rows of b, x), FP64."""
    A = _as_csr(A)
    b = np.atleast_2d(b)
    x = np.atleast_2d(x)
    r = b - (A @ x.T).T
    return np.linalg.norm(r, axis=1) / np.linalg.norm(b, axis=1)


def rms_error(x: np.ndarray, x_exact: np.ndarray) -> np.ndarray:
    """Root-mean-square error against the exact solution (the paper's metric, §7.1, §9)."""
    d = np.atleast_2d(x) - np.atleast_2d(x_exact)
    return np.sqrt(np.mean(d * d, axis=1))


def direct_solve(A, b: np.ndarray) -> np.ndarray:
    """Exact solution by a library sparse direct solve (the plain definition of A^{-1} b)."""
    import scipy.sparse.linalg as spla

    A = _as_csr(A).tocsc()
    b = np.atleast_2d(b)
    lu = spla.splu(A)
    return np.stack([lu.solve(bi) for bi in b])


@dataclass
class SolveResult:
    x: np.ndarray
    sweeps: int
    history: list
    state: State


def solve(split: SplitGraph, A, b: np.ndarray, Z, rtol: float = 1e-10, maxit: int = 10000,
          check_every: int = 1) -> SolveResult:
    """Iterate Table 1 from zero boundary variables until max relative residual <= rtol."""
    m = VTM(split, Z)
    b = np.atleast_2d(b)
    st = m.initial_state(b.shape[0])
    hist = []
    for k in range(1, maxit + 1):
        st = m.sweep(st, b)
        if k % check_every == 0 or k == maxit:
            x = m.assemble(st)
            rr = relative_residual(A, b, x)
            hist.append((k, float(np.max(rr))))
            if np.max(rr) <= rtol:
                return SolveResult(x=x, sweeps=k, history=hist, state=st)
    return SolveResult(x=m.assemble(st), sweeps=maxit, history=hist, state=st)


def residual_from_ports(split: SplitGraph, state: State) -> np.ndarray:
    """b - A x̄ of the assembled iterate (x̄ = mean of the copies) from port data alone, (R, n).

    KCL (Thm 4.1, App. 2) gives b - A x̄ = sum_j S_j (b̃_j - Ã_j x̄|_j), S_j the scatter of subgraph
    j's copies to their vertices.  Every local solve satisfies eq. 5.8, which with the current update
    reads Ã_j x_j = b̃_j + P_j omega_j (omega the inflow currents of the sweep), so

        b - A x̄ = sum_j S_j (Ã_j D_j - P_j omega_j),     D_j = x_j - x̄|_j.

    D_j vanishes on copies of vertices with one copy, so only the port potentials u, the currents
    omega and the columns of Ã_j at the ports are needed: no interior unknown.  This holds for the
    coupled lines of §7.2 as well (their current update keeps the same local equation)."""
    R = state.u.shape[0]
    xbar = assemble(split, state)                                   # mean of the copies
    out = np.zeros((R, split.n))
    piece_of_end = np.empty(2 * len(split.vtl), dtype=np.int64)
    local_of_end = np.empty(2 * len(split.vtl), dtype=np.int64)
    piece_of_end[0::2], local_of_end[0::2] = split.vtl[:, 0], split.vtl[:, 1]
    piece_of_end[1::2], local_of_end[1::2] = split.vtl[:, 2], split.vtl[:, 3]
    for j, g in enumerate(split.subgraphs):
        ends = np.nonzero(piece_of_end == j)[0]
        ports = np.unique(local_of_end[ends])
        D = np.zeros((R, len(g.vertices)))
        # D_j on the ports: the port potential of the copy (its u) minus the mean of the copies
        u_port = {}
        for e in ends:
            u_port[int(local_of_end[e])] = state.u[:, e]
        for c in ports:
            D[:, c] = u_port[int(c)] - xbar[:, g.vertices[c]]
        contrib = (g.A[:, ports] @ D[:, ports].T).T                   # Ã_j D_j: port columns only
        np.add.at(contrib.T, local_of_end[ends], -state.omega[:, ends].T)
        np.add.at(out.T, g.vertices, contrib.T)
    return out
