"""§9's qualitative claims on 2D grids (the paper's testbench shapes: (8 s + 1)^2 grids on 8 x 8
subgraphs, n = 4225 on p = 4 ... 64), as a regression of the FP64 oracle at Z = 1.  The paper says
the iteration count grows slowly with p and stays roughly flat in n.  Measured here: it grows
sublinearly in both, about p^0.48 at n = 4225 (285, 490, 975 sweeps for p = 4, 16, 64) and about
n^0.35 at p = 64 (395, 580, 975 sweeps for n = 289, 1089, 4225); flat in n is not reproduced at a
fixed Z = 1."""
import numpy as np

from oracle import evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def _sweeps(m, s):
    A = inputs.grid_poisson((m, m))
    split = evs.split_grid(A, (m, m), (s, s))
    b = inputs.rhs_uniform(A.n, 1, seed=0)
    r = ovtm.solve(split, A, b, 1.0, rtol=1e-8, maxit=20000, check_every=5)
    assert r.history[-1][1] <= 1e-8
    return r.sweeps


def test_section9_growth_in_p_and_n():
    k_p = [_sweeps(65, s) for s in (32, 16, 8)]          # n = 4225 on p = 4, 16, 64
    k_n = [_sweeps(8 * s + 1, s) for s in (2, 4)] + [k_p[-1]]   # p = 64, n = 289, 1089, 4225
    assert k_p[0] < k_p[1] < k_p[2] and k_p[2] / k_p[0] <= 1.25 * np.sqrt(64 / 4)
    assert k_n[0] < k_n[1] < k_n[2] and k_n[2] / k_n[0] <= np.sqrt(4225 / 289)
