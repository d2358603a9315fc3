"""Closed forms that pin the iteration (paper App. 3, §2, §7.1) — FP64 oracle.  TEST INFRASTRUCTURE ONLY.

1. Port-space operator of App. 3 (level-one splits only, as in the paper's proof).
   Order every port as seniors then juniors (one per line), eliminate the inner unknowns of the
   split system (eq. A3.2): S = blockdiag(C_se, C_ju) - [E_se; E_ju] D^{-1} [F_se F_ju]
   (eq. A3.3), M = diag(Z, Z), J the senior/junior exchange.  Then for k >= 2
       û^k = P û^{k-1} + γ,   P = (I + M S)^{-1} J (I - M S)            (eq. A3.8)
   so the port error e^k = û^k - û* obeys e^k = P e^{k-1} exactly, and Thm 6.1's convergence is
   spectral radius ρ(P) < 1.  (The relation needs omega^{k-1} = S û^{k-1} - β, which holds once
   one local solve has been done, hence k >= 2.)

2. One line between two subgraphs (level one, a single split vertex).  Seen from its port a
   subgraph is a Thevenin source: u = v + r_in * omega (Def. 7.1 gives r_in).  With the incident
   wave w_in = u_twin - Z omega_twin (right side of eq. 5.6) the port obeys u + Z omega = w_in,
   so the outgoing wave u - Z omega equals T v + Γ w_in with the reflection coefficient
       Γ = (r_in - Z) / (r_in + Z).
   Wave errors therefore contract by Γ_a Γ_b every two iterations, and a line matched to one
   side (Z = r_in of that side, Γ = 0) is exact after three iterations from any start.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .evs import SplitGraph


def port_operator(split: SplitGraph, Z) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Return (P, S, ports) of eq. A3.8 for a level-one split; ports[k] = (j, c) in û order."""
    m = len(split.vtl)
    Zl = np.broadcast_to(np.asarray(Z, dtype=np.float64), (m,))
    # global split system Ã = blockdiag(Ã_j), unknowns numbered subgraph by subgraph
    offs = np.cumsum([0] + [len(g.vertices) for g in split.subgraphs])
    Abar = sp.block_diag([g.A for g in split.subgraphs]).toarray()
    se = offs[split.vtl[:, 0]] + split.vtl[:, 1]
    ju = offs[split.vtl[:, 2]] + split.vtl[:, 3]
    ports = np.concatenate([se, ju])
    if len(np.unique(ports)) != len(ports):
        raise ValueError("port_operator needs a level-one split (one line per port)")
    inner = np.setdiff1d(np.arange(Abar.shape[0]), ports)
    C = Abar[np.ix_(ports, ports)]
    E = Abar[np.ix_(ports, inner)]
    F = Abar[np.ix_(inner, ports)]
    D = Abar[np.ix_(inner, inner)]
    S = C - E @ np.linalg.solve(D, F) if len(inner) else C          # eq. A3.3
    M = np.diag(np.concatenate([Zl, Zl]))
    I = np.eye(2 * m)
    J = np.block([[np.zeros((m, m)), np.eye(m)], [np.eye(m), np.zeros((m, m))]])
    P = np.linalg.solve(I + M @ S, J @ (I - M @ S))                  # eq. A3.8
    pl = [(int(j), int(c)) for j, c in zip(split.vtl[:, 0], split.vtl[:, 1])] + \
         [(int(j), int(c)) for j, c in zip(split.vtl[:, 2], split.vtl[:, 3])]
    return P, S, np.array(pl)


def spectral_radius(P: np.ndarray) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(P))))


def reflection_coefficient(r_in: float, Z: float) -> float:
    """Γ = (r_in - Z)/(r_in + Z) of a port with input impedance r_in on a line of impedance Z."""
    return (r_in - Z) / (r_in + Z)
