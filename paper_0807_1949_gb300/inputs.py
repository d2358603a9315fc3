"""Seeded synthetic problem generators shared by the tests, the benchmark and the oracle.

This module only builds the *problem* ``A x = b`` (an SPD matrix in symmetric CSR form and
right-hand sides).  It contains none of the arithmetic of Electric Vertex Splitting or of the
Virtual Transmission Method: splitting, local systems, waves and residuals live elsewhere.

Every generator is deterministic in its ``seed`` (numpy ``default_rng``).

Matrix format (the C ABI's ``vtm_csr``): full symmetric CSR, ``rowptr`` int64 of length n+1,
``col`` int32 sorted ascending within each row, ``val`` float64.
Right-hand sides: float64 array of shape ``(nrhs, n)`` (column-major n x nrhs, one RHS per
row of the numpy array).

Workloads (the paper's §9 testbenches are 2D grids cut into square blocks; §8's cost model
assumes a 2D grid on a 2D processor mesh):

* ``grid_poisson``: 2D 5-point / 3D 7-point variable-coefficient Poisson operator on a vertex
  grid with homogeneous Dirichlet conditions eliminated.  Node coefficient
  ``k_i = exp(sigma * N(0,1))``; edge weight between neighbours is the harmonic mean
  ``2 k_i k_j / (k_i + k_j)``; a missing neighbour outside the grid contributes ``k_i`` to the
  diagonal (Dirichlet).  ``sigma = 0`` gives the constant-coefficient Laplacian
  (diagonal 4 in 2D, 6 in 3D).
* ``random_dd_spd``: random sparse symmetric matrix with negative off-diagonals and a
  positive diagonal excess (weakly diagonally dominant, SPD).
* ``random_spd_dense``: dense random SPD matrix (tiny sizes) for theory tests.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Full symmetric CSR matrix (both triangles stored)."""

    n: int
    rowptr: np.ndarray  # int64, n+1
    col: np.ndarray     # int32, nnz
    val: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col.astype(np.int64), self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d


def _csr_from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    # merge duplicates
    key = rows.astype(np.int64) * n + cols
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n=n, rowptr=rowptr, col=c, val=sums.astype(np.float64))


def csr_from_dense(a: np.ndarray) -> CSR:
    a = np.asarray(a, dtype=np.float64)
    rows, cols = np.nonzero(a)
    return _csr_from_coo(a.shape[0], rows.astype(np.int64), cols.astype(np.int64), a[rows, cols])


def grid_poisson(dims, sigma: float = 0.0, seed: int = 0) -> CSR:
    """Variable-coefficient Poisson operator on a 2D or 3D vertex grid, Dirichlet eliminated.

    ``dims = (nx, ny)`` or ``(nx, ny, nz)``; vertex id ``i = x + nx*(y + ny*z)``.
    """
    dims = tuple(int(d) for d in dims)
    if len(dims) == 2:
        dims = dims + (1,)
    nx, ny, nz = dims
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    if sigma > 0:
        k = np.exp(sigma * rng.standard_normal(n))
    else:
        k = np.ones(n)
    idx = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    active = [a for a, d in enumerate((nx, ny, nz)) if d > 1]
    for axis in active:  # 0 = x, 1 = y, 2 = z
        np_axis = 2 - axis
        ext = (nx, ny, nz)[axis]
        lo = np.take(idx, np.arange(ext - 1), axis=np_axis).ravel()
        hi = np.take(idx, np.arange(1, ext), axis=np_axis).ravel()
        w = 2.0 * k[lo] * k[hi] / (k[lo] + k[hi])
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [-w, -w]
        np.add.at(diag, lo, w)
        np.add.at(diag, hi, w)
        # Dirichlet neighbours outside the grid on both faces of this axis
        first = np.take(idx, [0], axis=np_axis).ravel()
        last = np.take(idx, [ext - 1], axis=np_axis).ravel()
        np.add.at(diag, first, k[first])
        np.add.at(diag, last, k[last])
    rows.append(np.arange(n, dtype=np.int64))
    cols.append(np.arange(n, dtype=np.int64))
    vals.append(diag)
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def grid_anisotropic9(nx: int, ny: int, rho: float = 0.6) -> CSR:
    """-(u_xx + 2 rho u_xy + u_yy) on an nx x ny vertex grid, Dirichlet eliminated: the 9-point
    stencil with centre 4, axis neighbours -1 and diagonal neighbours -rho/2 (along x = y) and
    +rho/2 (along x = -y).  SPD for |rho| < 1, but a row's off-diagonal sum 4 + 2|rho| exceeds its
    diagonal: not diagonally dominant.  Vertex id i = x + nx*y."""
    idx = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(nx * ny, 4.0)]
    for dx, dy, v in ((1, 0, -1.0), (0, 1, -1.0), (1, 1, -0.5 * rho), (1, -1, 0.5 * rho)):
        ys = np.arange(max(0, -dy), ny - max(0, dy))
        xs = np.arange(0, nx - dx)
        a = idx[np.ix_(ys, xs)].ravel()
        b = idx[np.ix_(ys + dy, xs + dx)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(len(a), v), np.full(len(a), v)]
    return _csr_from_coo(nx * ny, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def random_dd_spd(n: int, avg_degree: float = 4.0, excess: float = 0.1, seed: int = 0) -> CSR:
    """Random sparse symmetric, weakly diagonally dominant matrix with positive excess (SPD).

    Off-diagonals are ``-U(0.1, 1)``; the diagonal is the row's absolute off-diagonal sum
    plus ``excess * U(0, 1)`` (at least 1e-3 so that the matrix is SPD even when a row has
    no neighbours).  A path through all vertices keeps the graph connected.
    """
    rng = np.random.default_rng(seed)
    m = int(n * avg_degree / 2)
    a = rng.integers(0, n, m)
    b = rng.integers(0, n, m)
    keep = a != b
    a, b = a[keep], b[keep]
    path_a = np.arange(n - 1)
    path_b = np.arange(1, n)
    a = np.concatenate([a, path_a])
    b = np.concatenate([b, path_b])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pairs = np.unique(lo.astype(np.int64) * n + hi)
    lo, hi = pairs // n, pairs % n
    w = rng.uniform(0.1, 1.0, len(lo))
    diag = np.zeros(n)
    np.add.at(diag, lo, w)
    np.add.at(diag, hi, w)
    diag += np.maximum(excess * rng.uniform(0.0, 1.0, n), 1e-3)
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    vals = np.concatenate([-w, -w, diag])
    return _csr_from_coo(n, rows, cols, vals)


def random_spd_dense(n: int, seed: int = 0, shift: float = 0.5) -> np.ndarray:
    """Dense random SPD matrix ``G G^T / n + shift I``."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n))
    return g @ g.T / n + shift * np.eye(n)


def rhs_uniform(n: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """Right-hand sides i.i.d. uniform[-1, 1]; shape ``(nrhs, n)`` float64."""
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(-1.0, 1.0, size=(nrhs, n))


def grid_coordinates(dims) -> np.ndarray:
    """Integer coordinates (n, 3) of the vertices of a grid in the generator's numbering."""
    dims = tuple(int(d) for d in dims)
    if len(dims) == 2:
        dims = dims + (1,)
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


@dataclass
class FEMProblem:
    """P1 finite elements on a Delaunay triangulation (the problem only, no splitting).

    A              assembled stiffness on the interior nodes (hull nodes are Dirichlet, eliminated)
    elem_nodes     (m, 3) int64 triangle vertices in the original node numbering
    elem_mats      (m, 3, 3) float64 element stiffness matrices k_e * area * grad(phi_a).grad(phi_b)
    node_unknown   (N,) int64: unknown index in A of each node, -1 for Dirichlet nodes
    centroids      (m, 2) float64 triangle centroids
    coords         (N, 2) float64 node coordinates
    """

    A: CSR
    elem_nodes: np.ndarray
    elem_mats: np.ndarray
    node_unknown: np.ndarray
    centroids: np.ndarray
    coords: np.ndarray


def fem_delaunay(npoints: int, pattern: int = 8, k_lo: float = 1e-3, k_hi: float = 1e3, seed: int = 0) -> FEMProblem:
    """P1 stiffness of -div(k grad u) on the Delaunay triangulation of uniform random points in the
    unit square, k a checkerboard of k_lo / k_hi on a pattern x pattern grid (by triangle centroid),
    homogeneous Dirichlet conditions on the convex hull."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(npoints, 2))
    tri = Delaunay(pts)
    T = tri.simplices.astype(np.int64)
    P = pts[T]                                             # (m, 3, 2)
    cen = P.mean(axis=1)
    cell = np.floor(np.clip(cen, 0, 1 - 1e-12) * pattern).astype(np.int64)
    k = np.where((cell[:, 0] + cell[:, 1]) % 2 == 0, k_lo, k_hi)
    # barycentric gradients: grad phi_a = perp(p_c - p_b) / (2 area) for (a, b, c) cyclic
    d = np.stack([P[:, 2] - P[:, 1], P[:, 0] - P[:, 2], P[:, 1] - P[:, 0]], axis=1)   # (m, 3, 2)
    area2 = d[:, 1, 0] * d[:, 2, 1] - d[:, 1, 1] * d[:, 2, 0]
    sign = np.sign(area2)[:, None, None]
    G = np.stack([-d[..., 1], d[..., 0]], axis=-1) * sign       # gradients times 2*area
    area = 0.5 * np.abs(area2)
    Ke = (k / (4.0 * area))[:, None, None] * np.einsum("mad,mbd->mab", G, G)
    hull = np.unique(tri.convex_hull.ravel())
    unknown = np.full(npoints, -1, dtype=np.int64)
    interior = np.setdiff1d(np.arange(npoints), hull)
    unknown[interior] = np.arange(len(interior))
    U = unknown[T]                                             # (m, 3)
    rows = np.repeat(U, 3, axis=1).ravel()
    cols = np.tile(U, (1, 3)).ravel()
    vals = Ke.reshape(len(T), 9).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = _csr_from_coo(len(interior), rows[keep], cols[keep], vals[keep])
    return FEMProblem(A=A, elem_nodes=T, elem_mats=Ke, node_unknown=unknown, centroids=cen, coords=pts)
