"""Pins of the general conformal split (oracle/conformal.py, App. 1, Thm 4.2) against the paper's
printed two-vertex construction, KCL, SPD-ness where the diagonal rule fails, the line tree of
every vertex, and convergence of Table 1 to the direct solution."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import conformal, evs
from oracle import vtm as ovtm
from paper_0807_1949_gb300 import inputs


def _block_home(nx, ny, bx, by):
    """Home subgraph of each vertex of an nx x ny grid cut into bx x by blocks (id x + nx y)."""
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    return ((x * bx) // nx + bx * ((y * by) // ny)).ravel()


def _scatter(split):
    n = split.n
    tot = np.zeros((n, n))
    shares = np.zeros(n)
    for g in split.subgraphs:
        tot[np.ix_(g.vertices, g.vertices)] += g.A.toarray()
        np.add.at(shares, g.vertices, g.share)
    return tot, shares


def test_app1_two_vertex_construction():
    """App. 1 step 2, x_2 on the boundary: the subgraph with the interior vertex x_1 is
    [[a11, a12], [a21, l a22 + (1 - l) a12^2 / a11]] and the other one (1 - l)(a22 - a12^2 / a11),
    l the paper's share.  Here x_1 is the beta interior, so l = 1 - lam."""
    a11, a12, a22 = 2.0, -1.7, 1.9          # SPD (det 0.91), |a12| > a22: not diagonally dominant
    A = np.array([[a11, a12], [a12, a22]])
    lam = 0.3
    s = conformal.split_conformal(sp.csr_matrix(A), home=[1, 0], lam=lam)
    l = 1.0 - lam
    alpha, beta = s.subgraphs                # alpha: the boundary copy of x_2 alone; beta: x_1, x_2
    assert list(alpha.vertices) == [1] and list(beta.vertices) == [0, 1]
    ref_beta = np.array([[a11, a12], [a12, l * a22 + (1 - l) * a12 ** 2 / a11]])
    ref_alpha = np.array([[(1 - l) * (a22 - a12 ** 2 / a11)]])
    assert np.allclose(beta.A.toarray(), ref_beta, rtol=0, atol=1e-15)
    assert np.allclose(alpha.A.toarray(), ref_alpha, rtol=0, atol=1e-15)
    assert len(s.vtl) == 1


@pytest.mark.parametrize("nx,ny,bx,by,rho", [(12, 10, 2, 2, 0.6), (16, 9, 4, 2, 0.9), (9, 9, 3, 1, 0.3)])
def test_kcl_and_spd_where_the_diagonal_rule_fails(nx, ny, bx, by, rho):
    A = inputs.grid_anisotropic9(nx, ny, rho)
    As = A.to_scipy()
    home = _block_home(nx, ny, bx, by)
    # the diagonal rule of evs.py cannot split this matrix
    owners = [tuple(sorted({int(home[i])} | {int(home[k]) for k in As.indices[As.indptr[i]:As.indptr[i + 1]]}))
              for i in range(A.n)]
    with pytest.raises(evs.NotConformal):
        evs.split_by_owners(As, owners, [])
    s = conformal.split_conformal(A, home, lam=0.35)    # lam != 1/2: the two shares of S differ
    assert len(s.subgraphs) == bx * by
    tot, shares = _scatter(s)
    assert np.max(np.abs(tot - As.toarray())) <= 1e-12 * np.abs(As).max()
    assert np.allclose(shares, 1.0, rtol=0, atol=1e-15)
    for g in s.subgraphs:
        assert np.linalg.eigvalsh(g.A.toarray()).min() > 0
        assert abs(g.A - g.A.T).max() <= 1e-13 * abs(g.A).max()
    # the copies of every vertex are joined by a tree of lines
    ncopies = np.zeros(A.n, dtype=int)
    for g in s.subgraphs:
        np.add.at(ncopies, g.vertices, 1)
    parent = {}

    def find(x):
        while parent.get(x, x) != x:
            x = parent[x]
        return x

    nlines = np.zeros(A.n, dtype=int)
    for pa, ca, pb, cb in s.vtl:
        v = s.subgraphs[pa].vertices[ca]
        assert v == s.subgraphs[pb].vertices[cb] and pa != pb
        nlines[v] += 1
        ra, rb = find((pa, ca)), find((pb, cb))
        assert ra != rb                      # no cycle
        parent[ra] = rb
    assert np.array_equal(nlines, ncopies - 1)


@pytest.mark.parametrize("lam", [0.5, 0.2])
def test_table1_on_the_conformal_split_converges(lam):
    """Thm 6.1 (SPD pieces, any Z > 0) and Thm 4.1: the VTM iteration on this split reaches the
    solution of A x = b."""
    A = inputs.grid_anisotropic9(14, 12, 0.7)
    s = conformal.split_conformal(A, _block_home(14, 12, 2, 2), lam=lam)
    b = inputs.rhs_uniform(A.n, 1, seed=3)
    r = ovtm.solve(s, A, b, 1.0, rtol=1e-10, maxit=4000, check_every=10)
    assert r.history[-1][1] <= 1e-10
    xs = ovtm.direct_solve(A, b)
    assert np.max(np.abs(r.x - xs)) <= 1e-8 * np.max(np.abs(xs))
