"""Impedance matching (paper §7.1) — FP64 oracle.  TEST INFRASTRUCTURE ONLY.

Def. 7.1: with all sources and all other inflow currents of a subgraph set to zero, a unit
inflow current at port c produces the potential u_c; that potential is the port's input
impedance r_in,c = u_c = (Ã_j^{-1})_{cc}.

A subgraph whose Ã_j is singular (an interior block of a Dirichlet problem: every row sums to
zero, Cor. 4.1 only guarantees SNND) has no input impedance in the sense of Def. 7.1.  The
reading used here (``terminate=True``): the other lines stay connected to their (matched)
transmission lines, i.e. every other end e' of the subgraph adds Z_{e'}^{-1} to its port's
diagonal, and so do the port's own other lines when it has several; the input impedance seen by
end e is then (K_e^{-1})_{cc} with K_e = K_j - Z_e^{-1} e_c e_c^T (K_j from eq. 5.8).

Matching rule (§7.1 asks for Z "near the input impedance of either port"; reading): the
geometric mean of the two ends' input impedances, Z_t = sqrt(r_in(a) * r_in(b)).

Pins: Example 7.1's four values (tests/golden/example_7_1.json) for the open definition; for the
terminated reading, brute-force Sherman-Morrison identity against the full termination, and a
one-port subgraph where both readings coincide.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .evs import SplitGraph
from .vtm import Ends, ends_of


def input_impedance_open(A_j, c: int) -> float:
    """Def. 7.1 literally: solve Ã_j x = e_c and return x_c."""
    Ad = A_j.toarray() if sp.issparse(A_j) else np.asarray(A_j, dtype=np.float64)
    e = np.zeros(Ad.shape[0])
    e[c] = 1.0
    return float(np.linalg.solve(Ad, e)[c])


def input_impedance_terminated(split: SplitGraph, ends: Ends, e: int) -> float:
    """Input impedance seen by end e with every other line of its subgraph terminated."""
    j, c = ends.piece[e], ends.local[e]
    K = split.subgraphs[j].A.toarray()
    for f in np.nonzero(ends.piece == j)[0]:
        if f != e:
            K[ends.local[f], ends.local[f]] += 1.0 / ends.Z[f]
    rhs = np.zeros(K.shape[0])
    rhs[c] = 1.0
    return float(np.linalg.solve(K, rhs)[c])


def matched_impedances(split: SplitGraph, Z0=1.0, terminate: bool = True) -> np.ndarray:
    """Z_t = sqrt(r_in(a) r_in(b)) for every line t (ends terminated with Z0 when needed)."""
    ends = ends_of(split, Z0)
    m = len(split.vtl)
    r = np.empty(2 * m)
    for e in range(2 * m):
        if terminate:
            r[e] = input_impedance_terminated(split, ends, e)
        else:
            r[e] = input_impedance_open(split.subgraphs[ends.piece[e]].A, ends.local[e])
    return np.sqrt(r[0::2] * r[1::2])
