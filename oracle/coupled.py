"""Coupled virtual transmission lines (paper §7.2, Thm 7.1) — FP64 oracle.  TEST INFRASTRUCTURE
ONLY.

§7.2 lets the local impedance Z_j of eq. 5.8 be a full symmetric matrix instead of a diagonal one:
the lines that leave subgraph j are then coupled, and Thm 7.1 states convergence whenever every
Z_j is SPD.  This module runs Table 1 with such matrices.

Reading (the paper gives the matrix but not its structure):

* Lines are coupled only inside a *bundle*: the set of lines that join the same two subgraphs.
  Both ends of a bundle see the same impedance matrix (one physical multi-conductor line), just
  as both ends of an uncoupled line share Z_t.  Lines of different bundles are never coupled, so
  Z_j is block diagonal over the bundles that reach subgraph j.
* The coupling is given by the admittance matrix Y = Z^{-1} over all lines (sparse, symmetric,
  SPD, zero between lines of different bundles); Y = diag(1/Z_t) is the uncoupled method.

With the end's potential u and inflow current omega of §5 (vectors over the lines at subgraph j,
in end order), eq. 5.6 for a bundle reads u_j^k + Z omega_j^k = u_twin^{k-1} - Z omega_twin^{k-1}.
Solving it for omega_j^k and putting that into the KCL of subgraph j gives eq. 5.8 with the
matrix impedance:

    K_j = Ã_j + P_j Y_j P_j^T,      r_j = b̃_j + P_j (Y_j u_twin^{k-1} - omega_twin^{k-1}),
    omega_j^k = Y_j (u_twin^{k-1} - u_j^k) - omega_twin^{k-1},

where P_j maps the ends at j to their local unknowns and Y_j is Y restricted to the lines at j.
No matrix is ever inverted: the iteration needs Y only.  The outgoing wave u - Z omega, which
does need Z = Y^{-1}, is formed per bundle by ``waves_out`` for the closed-form pins.

Pins (tests/test_oracle_coupled.py): Y diagonal reproduces the uncoupled oracle; Thm 7.1 (random
SPD bundle admittances converge to the direct solution); Thm 4.1 at the fixed point (twins equal,
currents opposite); the multi-conductor reflection law, i.e. the wave error leaving subgraph a is
Gamma_a = (R_a - Z)(R_a + Z)^{-1} times the error arriving there, R_a = P^T Ã_a^{-1} P the input
impedance matrix of Def. 7.1 taken over a whole bundle; and the matched bundle Z = R_a (so
Gamma_a = 0), which is exact after three sweeps.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .evs import SplitGraph, _as_csr
from .vtm import BandedCholesky, State


def bundles(split: SplitGraph) -> dict:
    """Bundle of every line: key (min piece, max piece) -> array of line ids."""
    out: dict = {}
    for t, (ja, _, jb, _) in enumerate(split.vtl):
        out.setdefault((min(ja, jb), max(ja, jb)), []).append(t)
    return {k: np.asarray(v, dtype=np.int64) for k, v in out.items()}


def laplacian_admittance(split: SplitGraph, Z, pairs, y) -> sp.csr_matrix:
    """Y = diag(1/Z_t) + sum_p y_p (e_t - e_t')(e_t - e_t')^T for line pairs p = (t, t'): a
    conductance y_p >= 0 between two lines of one bundle.  SPD for Z > 0 and y >= 0."""
    m = len(split.vtl)
    Zl = np.broadcast_to(np.asarray(Z, dtype=np.float64), (m,))
    Y = sp.lil_matrix((m, m))
    Y.setdiag(1.0 / Zl)
    for (t, u), v in zip(np.asarray(pairs, dtype=np.int64).reshape(-1, 2), np.broadcast_to(y, (len(pairs),))):
        Y[t, t] += v
        Y[u, u] += v
        Y[t, u] -= v
        Y[u, t] -= v
    return Y.tocsr()


def local_matrix(A_j: sp.spmatrix, local: np.ndarray, Yj: np.ndarray) -> sp.csr_matrix:
    """K_j = Ã_j + P_j Y_j P_j^T (eq. 5.8 with the matrix Z_j), P_j[local[e], e] = 1."""
    n = A_j.shape[0]
    P = sp.csr_matrix((np.ones(len(local)), (local, np.arange(len(local)))), shape=(n, len(local)))
    return (A_j + P @ sp.csr_matrix(Yj) @ P.T).tocsr()


def inflow(u_twin: np.ndarray, omega_twin: np.ndarray, Yj: np.ndarray) -> np.ndarray:
    """Port current injected by the incoming waves, Y_j u_twin - omega_twin = Y_j w_in (R, ends)."""
    return u_twin @ Yj - omega_twin


def current_update(u_twin: np.ndarray, omega_twin: np.ndarray, u_new: np.ndarray, Yj: np.ndarray) -> np.ndarray:
    """omega_j^k = Y_j (u_twin^{k-1} - u_j^k) - omega_twin^{k-1} (eq. 5.6 solved for omega)."""
    return (u_twin - u_new) @ Yj - omega_twin


class CoupledVTM:
    """Table 1 with the bundle admittance matrix Y (module docstring)."""

    def __init__(self, split: SplitGraph, Y):
        self.split = split
        Y = sp.csr_matrix(Y, dtype=np.float64)
        m = len(split.vtl)
        if Y.shape != (m, m):
            raise ValueError("Y must be nlines x nlines")
        if abs(Y - Y.T).max() > 0:
            raise ValueError("Y must be symmetric")
        key = {}
        for k, ts in bundles(split).items():
            for t in ts:
                key[int(t)] = k
        Yc = Y.tocoo()
        for t, u in zip(Yc.row, Yc.col):
            if key[int(t)] != key[int(u)]:
                raise ValueError(f"lines {t} and {u} join different pairs of subgraphs")
        self.Y = Y
        npc = len(split.subgraphs)
        # ends: 2t = side a of line t, 2t+1 = side b; twin(e) = e ^ 1
        self.end_piece = np.empty(2 * m, dtype=np.int64)
        self.end_local = np.empty(2 * m, dtype=np.int64)
        self.end_piece[0::2], self.end_local[0::2] = split.vtl[:, 0], split.vtl[:, 1]
        self.end_piece[1::2], self.end_local[1::2] = split.vtl[:, 2], split.vtl[:, 3]
        self.ends_at = [np.nonzero(self.end_piece == j)[0] for j in range(npc)]
        self.Yj = [Y[self.ends_at[j] >> 1][:, self.ends_at[j] >> 1].toarray() for j in range(npc)]
        self.factor = {j: BandedCholesky(local_matrix(split.subgraphs[j].A, self.end_local[self.ends_at[j]],
                                                      self.Yj[j])) for j in range(npc)}

    def initial_state(self, nrhs: int = 1) -> State:
        E = len(self.end_piece)
        return State(u=np.zeros((nrhs, E)), omega=np.zeros((nrhs, E)), x_local=[None] * len(self.split.subgraphs))

    def sweep(self, state: State, b: np.ndarray) -> State:
        """One synchronous iteration over all subgraphs (Table 1 steps 3-5, matrix Z_j)."""
        b = np.atleast_2d(b)
        new_u = state.u.copy()
        new_om = state.omega.copy()
        x_local = list(state.x_local)
        for j in range(len(self.split.subgraphs)):
            e = self.ends_at[j]
            tw = e ^ 1
            r = self.split.local_rhs(b, j).copy()
            np.add.at(r.T, self.end_local[e], inflow(state.u[:, tw], state.omega[:, tw], self.Yj[j]).T)
            x = self.factor[j].solve(r)
            x_local[j] = x
            new_u[:, e] = x[:, self.end_local[e]]
            new_om[:, e] = current_update(state.u[:, tw], state.omega[:, tw], new_u[:, e], self.Yj[j])
        return State(u=new_u, omega=new_om, x_local=x_local)

    def waves_out(self, state: State) -> np.ndarray:
        """Outgoing wave u - Z omega of every end, Z = Y^{-1} per bundle; (R, E)."""
        w = state.u.copy()
        for ts in bundles(self.split).values():
            Zb = np.linalg.inv(self.Y[ts][:, ts].toarray())
            for side in (0, 1):
                e = 2 * ts + side
                w[:, e] -= state.omega[:, e] @ Zb
        return w

    def assemble(self, state: State) -> np.ndarray:
        """x_i = mean of the copies of vertex i (the uncoupled oracle's reading); (R, n)."""
        R = state.u.shape[0]
        acc = np.zeros((R, self.split.n))
        cnt = np.zeros(self.split.n)
        for j, g in enumerate(self.split.subgraphs):
            if state.x_local[j] is None:
                continue
            np.add.at(acc.T, g.vertices, state.x_local[j].T)
            np.add.at(cnt, g.vertices, 1.0)
        return acc / np.maximum(cnt, 1.0)[None, :]


def adjacent_line_pairs(split: SplitGraph, A=None) -> tuple[np.ndarray, np.ndarray]:
    """Pairs (t, t'), t < t', of lines of one bundle whose copies are neighbours in both subgraphs
    (an off-diagonal entry of Ã_j joins them on each side), and |a_ik| of the original matrix for
    the vertices i, k of the two lines (the sum of that edge's shares over the subgraphs)."""
    pairs, wts = [], []
    As = None if A is None else _as_csr(A)
    for (ja, jb), ts in bundles(split).items():
        at = {}
        for t in ts:
            va, ca, vb, cb = split.vtl[t]
            la, lb = (ca, cb) if va == ja else (cb, ca)
            at[(ja, int(la))] = int(t)
            at[(jb, int(lb))] = int(t)
        Aa = split.subgraphs[ja].A.tocsr()
        Ab = split.subgraphs[jb].A.tocsr()
        for t in ts:
            va, ca, vb, cb = split.vtl[t]
            la, lb = (ca, cb) if va == ja else (cb, ca)
            for k in Aa.indices[Aa.indptr[la]:Aa.indptr[la + 1]]:
                u = at.get((ja, int(k)))
                if u is None or u <= t:
                    continue
                va2, ca2, vb2, cb2 = split.vtl[u]
                lb2 = cb2 if va2 == ja else ca2
                if Ab[lb, lb2] == 0:
                    continue
                i = split.subgraphs[ja].vertices[la]
                i2 = split.subgraphs[ja].vertices[k]
                w = abs(Aa[la, k]) + abs(Ab[lb, lb2]) if As is None else abs(As[i, i2])
                pairs.append((int(t), u))
                wts.append(float(w))
    return np.asarray(pairs, dtype=np.int64).reshape(-1, 2), np.asarray(wts)
