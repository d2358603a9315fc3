"""Conformal splitting of a general SPD matrix (paper App. 1: Lemma A1.1, Thm 4.2) — FP64 oracle.
TEST INFRASTRUCTURE ONLY.

The split of evs.py needs weak diagonal dominance at the boundary vertices (step 3's diagonal
rule).  App. 1 proves that any SPD graph can be split into two SPD subgraphs at any boundary, by
completing the square over the vertices that are not on the boundary, and into N subgraphs by
repeating the split (Thm 4.2).  This module builds that split.

One split of a subgraph with SPD matrix M over copies V (App. 1 steps 2-4, in block form): the
copies are divided into an alpha side and a beta side; the boundary B is the set of alpha copies
that M joins to a beta copy, so that no entry of M joins the alpha interior I_a = alpha \\ B to the
beta interior I_b = beta.  Completing the square over each interior,

    x^T M x = (I_a part)^2 + (I_b part)^2 + x_B^T S x_B,
    S = M_BB - M_Ba M_aa^{-1} M_aB - M_Bb M_bb^{-1} M_bB          (SPD: a Schur complement of M),

and the boundary copies are split (variable splitting, App. 1 eq. A1.2) so that the alpha copy
keeps the fraction lam of S and the beta copy the rest:

    M_alpha = [[M_aa, M_aB], [M_Ba, M_Ba M_aa^{-1} M_aB + lam S]]
    M_beta  = [[M_bb, M_bB], [M_Bb, M_Bb M_bb^{-1} M_bB + (1 - lam) S]]

Both are SPD for 0 < lam < 1 (their Schur complements on B are lam S and (1 - lam) S) and they sum
back to M on the merged variables (Thm 4.1).  For n = 2 with x_2 on the boundary this is the
printed construction of App. 1 step 2 (tests/test_oracle_conformal.py checks it).  Each boundary
copy's source share is divided in the same ratio, and one line joins the two copies.

N subgraphs (Thm 4.2: N - 1 splits): every vertex has a home subgraph; the ids [lo, hi) of a
subgraph being split are halved at mid = (lo + hi) / 2, alpha = copies whose home is below mid.  A
new beta copy takes as its home the smallest home among its beta neighbours.  The alpha copy keeps
the lines it already had.  The matrices are dense (the boundary blocks fill in): small problems.

Pins: App. 1 step 2 closed form; KCL (pieces sum to A, shares to 1); every piece SPD on a matrix
that is not diagonally dominant (where evs.py's rule fails); the lines of each vertex form a tree;
Table 1 on this split converges to the direct solution (Thm 6.1 needs SNND pieces only).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .evs import SplitGraph, Subgraph, _as_csr


def schur_terms(M, Ia, Ib, B):
    """T_a = M_Ba M_aa^{-1} M_aB, T_b = M_Bb M_bb^{-1} M_bB and S = M_BB - T_a - T_b (App. 1
    step 4: completing the square over each interior)."""
    MaB, MbB = M[np.ix_(Ia, B)], M[np.ix_(Ib, B)]
    Ta = MaB.T @ np.linalg.solve(M[np.ix_(Ia, Ia)], MaB) if Ia else np.zeros((len(B), len(B)))
    Tb = MbB.T @ np.linalg.solve(M[np.ix_(Ib, Ib)], MbB) if Ib else np.zeros((len(B), len(B)))
    return Ta, Tb, M[np.ix_(B, B)] - Ta - Tb


def boundary_blocks(Ta, Tb, S, lam):
    """The boundary blocks of the two new subgraphs: T_a + lam S and T_b + (1 - lam) S."""
    return Ta + lam * S, Tb + (1.0 - lam) * S


def split_conformal(A, home, lam: float = 0.5) -> SplitGraph:
    """Recursive App. 1 split of SPD ``A`` into ``max(home) + 1`` SPD subgraphs (module docstring)."""
    if not 0.0 < lam < 1.0:
        raise ValueError("lam must lie in (0, 1)")
    M0 = _as_csr(A).toarray()
    n = M0.shape[0]
    home = np.asarray(home, dtype=np.int64)
    N = int(home.max()) + 1
    if np.any(np.bincount(home, minlength=N) == 0):
        raise ValueError("every subgraph needs a home vertex")
    cvert = list(range(n))          # parent vertex of each copy
    chome = list(int(h) for h in home)
    cshare = [1.0] * n
    lines = []                      # pairs of copy ids
    pieces = [None] * N             # (copy ids, matrix)

    def rec(ids, M, lo, hi):
        if hi - lo == 1:
            pieces[lo] = (ids, M)
            return
        mid = (lo + hi) // 2
        a_side = [k for k, c in enumerate(ids) if chome[c] < mid]
        b_side = [k for k, c in enumerate(ids) if chome[c] >= mid]
        nz = M != 0.0
        B = [k for k in a_side if nz[k, b_side].any()]
        Bset = set(B)
        Ia = [k for k in a_side if k not in Bset]
        Ib = b_side
        Maa, MaB = M[np.ix_(Ia, Ia)], M[np.ix_(Ia, B)]
        Mbb, MbB = M[np.ix_(Ib, Ib)], M[np.ix_(Ib, B)]
        Ba, Bb = boundary_blocks(*schur_terms(M, Ia, Ib, B), lam)
        new = []
        for k in B:
            c = ids[k]
            nb = [chome[ids[q]] for q in b_side if nz[k, q]]
            cvert.append(cvert[c])
            chome.append(min(nb))
            cshare.append((1.0 - lam) * cshare[c])
            cshare[c] *= lam
            new.append(len(cvert) - 1)
            lines.append((c, len(cvert) - 1))
        Ma = np.block([[Maa, MaB], [MaB.T, Ba]])
        Mb = np.block([[Mbb, MbB], [MbB.T, Bb]])
        rec([ids[k] for k in Ia] + [ids[k] for k in B], Ma, lo, mid)
        rec([ids[k] for k in Ib] + new, Mb, mid, hi)

    rec(list(range(n)), M0, 0, N)
    where = {}
    subs = []
    for j, (ids, M) in enumerate(pieces):
        order = np.argsort([cvert[c] for c in ids], kind="stable")   # local order: ascending vertex
        ids = [ids[k] for k in order]
        M = M[np.ix_(order, order)]
        for loc, c in enumerate(ids):
            where[c] = (j, loc)
        subs.append(Subgraph(vertices=np.array([cvert[c] for c in ids], dtype=np.int64),
                             A=sp.csr_matrix(M), share=np.array([cshare[c] for c in ids])))
    vtl = np.array([(*where[a], *where[b]) for a, b in lines], dtype=np.int64).reshape(-1, 4)
    return SplitGraph(n=n, subgraphs=subs, vtl=vtl)
