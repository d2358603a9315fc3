"""Electric Vertex Splitting (paper §4, App. 2) — FP64 oracle.  TEST INFRASTRUCTURE ONLY.

The paper leaves the split shares open ("plenty of ways", §4) and proves that conformal schemes
exist (Thm 4.2, Cor. 4.1).  This oracle implements the reading used throughout the project:

* Step 1 (boundary): vertex i is a boundary vertex iff its owner set O(i) -- the subgraphs that
  contain a copy of i -- has two or more members.
* Step 2 (twins / children): one copy of i per member of O(i).
* Step 3 (split weights and sources):
    - edge (i, j), i != j, is given to every subgraph in O(i) ∩ O(j) with weight
      a_ij / |O(i) ∩ O(j)|  (edges touching an inner vertex are therefore not split);
    - the weight of a boundary vertex copy c of i is
      a_ii^(c) = sum_{j != i} |a_ij^(c)| + delta_i / |O(i)|,  delta_i = a_ii - sum_{j != i} |a_ij|,
      which needs delta_i >= 0 (weak diagonal dominance at boundary vertices); a delta_i that is
      negative only by rounding (|delta_i| <= 64 eps a_ii) is taken as zero; inner vertices
      keep a_ii unchanged;
    - the source of copy c is b_i / |O(i)|.
  Every subgraph is then weakly diagonally dominant, hence SNND (Cor. 4.1), and the pieces sum
  back to A and b (App. 2: C_se + C_ju = C, E_se + E_ju = E, f_se + f_ju = f).
* Step 4 (inflow currents): one virtual transmission line (VTL) per pair of copies that face each
  other.  Level one (two copies) gives one line; for grid blocks the multilevel topology of
  Fig. 7 is the hypercube: copies are joined when their blocks differ along exactly one axis
  (2 lines per copy at a 2D corner, 3 at a 3D corner).
* An explicit split (any conformal scheme, e.g. Example 4.1's uneven shares) can be given
  directly as a list of subgraphs.

Grid blocks: along an axis of extent m, cut lines are shared at coordinates s, 2s, ...; block q
covers [q*s, min((q+1)*s, m-1)], there are ceil((m-1)/s) blocks (one block when m == 1).
Subgraph id of block (qx, qy, qz) is qx + Bx*(qy + By*qz).  Local order within a subgraph:
ascending global vertex id.

Pins: Example 4.1/4.2 matrices and sources exactly (tests/golden/example_4_1.json);
KCL sums back to A and b; pieces SNND (eigenvalues); hypercube line counts of Fig. 7.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Subgraph:
    """One subgraph M_j: local unknowns, local matrix Ã_j and source shares (eq. 4.4)."""

    vertices: np.ndarray          # global vertex of each local unknown, local order
    A: sp.csr_matrix              # Ã_j (local, symmetric)
    share: np.ndarray             # b̃_j = share * b[vertices]
    b_explicit: np.ndarray | None = None  # explicit b̃_j (Example 4.1), overrides share*b


@dataclass
class SplitGraph:
    """The split electric graph G̃_e: subgraphs plus the VTL list.

    ``vtl[t] = (j_a, c_a, j_b, c_b)``: line t joins local unknown c_a of subgraph j_a with
    local unknown c_b of subgraph j_b.
    """

    n: int
    subgraphs: list[Subgraph]
    vtl: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), dtype=np.int64))

    def local_rhs(self, b: np.ndarray, j: int) -> np.ndarray:
        """b̃_j for a right-hand side b of shape (n,) or (R, n); returns (R, n_j)."""
        g = self.subgraphs[j]
        b2 = np.atleast_2d(b)
        if g.b_explicit is not None:
            return np.atleast_2d(g.b_explicit).astype(np.float64)
        return b2[:, g.vertices] * g.share[None, :]


class NotConformal(ValueError):
    """Step 3 cannot make the boundary copy weakly diagonally dominant (delta_i < 0)."""


def _excess(a_ii: float, offabs: float) -> float:
    """delta_i = a_ii - sum_{j != i} |a_ij| of a boundary vertex; rounding-level negatives are 0."""
    delta = a_ii - offabs
    if delta < 0:
        if delta >= -64 * np.finfo(np.float64).eps * abs(a_ii):
            return 0.0
        raise NotConformal(f"boundary vertex with a_ii={a_ii} is not weakly diagonally dominant")
    return delta


def _as_csr(A) -> sp.csr_matrix:
    if hasattr(A, "to_scipy"):
        return A.to_scipy().tocsr()
    if sp.issparse(A):
        return A.tocsr()
    return sp.csr_matrix(np.asarray(A, dtype=np.float64))


def split_by_owners(A, owners: list[tuple[int, ...]], vtl_pairs: list[tuple[int, int, int]]) -> SplitGraph:
    """EVS steps 1-4 for given owner sets.

    owners[i]    -- sorted tuple of subgraph ids that hold a copy of vertex i (step 1-2).
    vtl_pairs    -- (vertex i, subgraph p, subgraph q): a line between the copies of i in p, q.
    """
    A = _as_csr(A)
    n = A.shape[0]
    npieces = 1 + max(max(o) for o in owners)
    verts = [[] for _ in range(npieces)]
    for i in range(n):
        for p in owners[i]:
            verts[p].append(i)
    local = [dict() for _ in range(npieces)]
    for p in range(npieces):
        for c, i in enumerate(verts[p]):
            local[p][i] = c
    rows = [[] for _ in range(npieces)]
    cols = [[] for _ in range(npieces)]
    vals = [[] for _ in range(npieces)]
    Acoo = A.tocoo()
    offabs = np.zeros(n)
    diag = A.diagonal()
    for i, j, a in zip(Acoo.row, Acoo.col, Acoo.data):
        if i != j:
            offabs[i] += abs(a)
    # step 3: edges
    abs_in_piece = [dict() for _ in range(npieces)]
    for i, j, a in zip(Acoo.row, Acoo.col, Acoo.data):
        if i == j:
            continue
        common = sorted(set(owners[i]) & set(owners[j]))
        if not common:
            raise ValueError(f"edge ({i},{j}) lies in no subgraph")
        for p in common:
            share = a / len(common)
            rows[p].append(local[p][i])
            cols[p].append(local[p][j])
            vals[p].append(share)
            abs_in_piece[p][i] = abs_in_piece[p].get(i, 0.0) + abs(share)
    # step 3: vertex weights
    for i in range(n):
        o = owners[i]
        if len(o) == 1:
            p = o[0]
            rows[p].append(local[p][i]); cols[p].append(local[p][i]); vals[p].append(diag[i])
            continue
        delta = _excess(diag[i], offabs[i])
        for p in o:
            w = abs_in_piece[p].get(i, 0.0) + delta / len(o)
            rows[p].append(local[p][i]); cols[p].append(local[p][i]); vals[p].append(w)
    subs = []
    for p in range(npieces):
        m = len(verts[p])
        Ap = sp.csr_matrix((vals[p], (rows[p], cols[p])), shape=(m, m))
        v = np.array(verts[p], dtype=np.int64)
        share = np.array([1.0 / len(owners[i]) for i in verts[p]])
        subs.append(Subgraph(vertices=v, A=Ap, share=share))
    # step 4: lines
    vtl = np.array([(p, local[p][i], q, local[q][i]) for (i, p, q) in vtl_pairs], dtype=np.int64).reshape(-1, 4)
    return SplitGraph(n=n, subgraphs=subs, vtl=vtl)


def grid_axis_blocks(m: int, s: int) -> list[tuple[int, ...]]:
    """For each coordinate 0..m-1 of one axis, the blocks whose closed range contains it."""
    nb = max(1, -(-(m - 1) // s)) if m > 1 else 1
    out = []
    for c in range(m):
        bs = tuple(q for q in range(nb) if q * s <= c <= min((q + 1) * s, m - 1))
        out.append(bs)
    return out


def grid_owners(dims, block) -> tuple[list[tuple[int, ...]], list[tuple[int, int, int]], tuple[int, int, int]]:
    """Owner sets and hypercube lines (Fig. 7) for a grid cut into blocks with shared cut lines."""
    dims = tuple(dims) + (1,) * (3 - len(dims))
    block = tuple(block) + (1,) * (3 - len(block))
    per_axis = [grid_axis_blocks(dims[a], block[a]) for a in range(3)]
    nblk = tuple(1 + max(max(t) for t in per_axis[a]) for a in range(3))
    nx, ny, nz = dims
    owners, pairs = [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                combos = list(itertools.product(per_axis[0][x], per_axis[1][y], per_axis[2][z]))
                ids = sorted(q[0] + nblk[0] * (q[1] + nblk[1] * q[2]) for q in combos)
                owners.append(tuple(ids))
                for qa, qb in itertools.combinations(combos, 2):
                    if sum(1 for a in range(3) if qa[a] != qb[a]) == 1:
                        pa = qa[0] + nblk[0] * (qa[1] + nblk[1] * qa[2])
                        pb = qb[0] + nblk[0] * (qb[1] + nblk[1] * qb[2])
                        pairs.append((i, min(pa, pb), max(pa, pb)))
    return owners, pairs, nblk


def split_grid(A, dims, block) -> SplitGraph:
    """EVS of a grid operator into blocks (shared cut lines/planes), hypercube lines."""
    owners, pairs, _ = grid_owners(dims, block)
    return split_by_owners(A, owners, pairs)


def split_grid_piece(A, dims, block, piece: int):
    """Step 1-3 restricted to one grid subgraph (for sampled checks on large grids).

    Returns (vertices, Ã_j, share) of subgraph ``piece`` computed exactly as ``split_grid``
    would, without building the other subgraphs.
    """
    A = _as_csr(A)
    dims = tuple(dims) + (1,) * (3 - len(dims))
    block = tuple(block) + (1,) * (3 - len(block))
    per_axis = [grid_axis_blocks(dims[a], block[a]) for a in range(3)]
    nblk = tuple(1 + max(max(t) for t in per_axis[a]) for a in range(3))
    q = (piece % nblk[0], (piece // nblk[0]) % nblk[1], piece // (nblk[0] * nblk[1]))
    rng = [[c for c in range(dims[a]) if q[a] in per_axis[a][c]] for a in range(3)]
    nx, ny = dims[0], dims[1]
    zz, yy, xx = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    verts = (xx + nx * (yy + ny * zz)).ravel().astype(np.int64)
    verts.sort()
    coords = lambda v: (v % nx, (v // nx) % ny, v // (nx * ny))

    def owner_axes(v):
        x, y, z = coords(v)
        return per_axis[0][x], per_axis[1][y], per_axis[2][z]

    def n_owners(v):
        a, b, c = owner_axes(v)
        return len(a) * len(b) * len(c)

    def n_common(v, w):
        av, aw = owner_axes(v), owner_axes(w)
        cnt = 1
        for t in range(3):
            cnt *= len(set(av[t]) & set(aw[t]))
        return cnt

    local = {int(v): c for c, v in enumerate(verts)}
    rows, cols, vals = [], [], []
    diag = A.diagonal()
    for c, v in enumerate(verts):
        v = int(v)
        lo, hi = A.indptr[v], A.indptr[v + 1]
        offabs = 0.0
        inpiece = 0.0
        for j, a in zip(A.indices[lo:hi], A.data[lo:hi]):
            j = int(j)
            if j == v:
                continue
            offabs += abs(a)
            if j in local:
                share = a / n_common(v, j)
                rows.append(c); cols.append(local[j]); vals.append(share)
                inpiece += abs(share)
        no = n_owners(v)
        if no == 1:
            w = diag[v]
        else:
            w = inpiece + _excess(diag[v], offabs) / no
        rows.append(c); cols.append(c); vals.append(w)
    m = len(verts)
    Ap = sp.csr_matrix((vals, (rows, cols)), shape=(m, m))
    share = np.array([1.0 / n_owners(int(v)) for v in verts])
    return verts, Ap, share


def kcl_residual(split: SplitGraph, A) -> float:
    """max |sum_j P_j Ã_j P_j^T - A| (App. 2 identities), P_j mapping local to global."""
    A = _as_csr(A)
    tot = sp.csr_matrix(A.shape)
    for g in split.subgraphs:
        m = len(g.vertices)
        P = sp.csr_matrix((np.ones(m), (g.vertices, np.arange(m))), shape=(split.n, m))
        tot = tot + P @ g.A @ P.T
    d = (tot - A).tocoo()
    return float(np.max(np.abs(d.data))) if d.nnz else 0.0


def grid_piece_line_count(dims, block, piece: int) -> np.ndarray:
    """Number of lines at each local copy of a grid subgraph (hypercube rule of Fig. 7).

    A copy has one line per axis along which its vertex is shared by two blocks.
    Local order: ascending global vertex id, as in ``split_grid_piece``.
    """
    dims = tuple(dims) + (1,) * (3 - len(dims))
    block = tuple(block) + (1,) * (3 - len(block))
    per_axis = [grid_axis_blocks(dims[a], block[a]) for a in range(3)]
    nblk = tuple(1 + max(max(t) for t in per_axis[a]) for a in range(3))
    q = (piece % nblk[0], (piece // nblk[0]) % nblk[1], piece // (nblk[0] * nblk[1]))
    rng = [[c for c in range(dims[a]) if q[a] in per_axis[a][c]] for a in range(3)]
    zz, yy, xx = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
    cnt = np.zeros(xx.size, dtype=np.int64)
    for a, coord in enumerate((xx.ravel(), yy.ravel(), zz.ravel())):
        cnt += np.array([len(per_axis[a][c]) == 2 for c in coord], dtype=np.int64)
    return cnt


def rcb(coords: np.ndarray, nparts: int) -> np.ndarray:
    """Recursive coordinate bisection: split at position floor(|E| floor(p/2) / p) of the order by
    (coordinate, id) along the axis of largest extent; the first part gets the lower ids."""
    coords = np.asarray(coords, dtype=np.float64)
    piece = np.zeros(len(coords), dtype=np.int64)

    def rec(ids, p, base):
        if p <= 1:
            piece[ids] = base
            return
        pl = p // 2
        ext = coords[ids].max(axis=0) - coords[ids].min(axis=0)
        axis = int(np.argmax(ext))
        order = ids[np.lexsort((ids, coords[ids, axis]))]
        m = (len(ids) * pl) // p
        rec(order[:m], pl, base)
        rec(order[m:], p - pl, base + pl)

    rec(np.arange(len(coords)), nparts, 0)
    return piece


def split_by_elements(A, elem_nodes, elem_mats, node_unknown, elem_piece) -> SplitGraph:
    """EVS on the physical level (§4): each element goes to one subgraph, Ã_j = sum of its elements'
    matrices (SPSD each, so every piece is SNND, Cor. 4.1), b_i shared as b_i / |O(i)|.  Lines join
    the copies of vertex i in p and q when an element edge through i has elements of p and q around
    it.  Local order: ascending vertex.  Line order: sorted (vertex, p, q)."""
    A = _as_csr(A)
    n = A.shape[0]
    elem_nodes = np.asarray(elem_nodes)
    k = elem_nodes.shape[1]
    npieces = int(np.max(elem_piece)) + 1
    U = np.asarray(node_unknown)[elem_nodes]
    subs, local = [], []
    ncop = np.zeros(n, dtype=np.int64)
    for j in range(npieces):
        es = np.nonzero(elem_piece == j)[0]
        verts = np.unique(U[es][U[es] >= 0])
        ncop[verts] += 1
        local.append({int(v): c for c, v in enumerate(verts)})
        subs.append((es, verts))
    out = []
    for j, (es, verts) in enumerate(subs):
        rows, cols, vals = [], [], []
        for e in es:
            for a in range(k):
                for b in range(k):
                    ua, ub = U[e, a], U[e, b]
                    if ua >= 0 and ub >= 0:
                        rows.append(local[j][int(ua)]); cols.append(local[j][int(ub)]); vals.append(elem_mats[e][a][b])
        m = len(verts)
        Aj = sp.coo_matrix((vals, (rows, cols)), shape=(m, m)).tocsr()
        out.append(Subgraph(vertices=verts.astype(np.int64), A=Aj, share=1.0 / ncop[verts]))
    edge_pieces = {}
    for e in range(len(elem_nodes)):
        for a in range(k):
            for b in range(a + 1, k):
                u, v = sorted((int(elem_nodes[e, a]), int(elem_nodes[e, b])))
                edge_pieces.setdefault((u, v), set()).add(int(elem_piece[e]))
    trip = set()
    for (u, v), ps in edge_pieces.items():
        if len(ps) < 2:
            continue
        ps = sorted(ps)
        for node in (u, v):
            x = int(node_unknown[node])
            if x < 0:
                continue
            for i1 in range(len(ps)):
                for i2 in range(i1 + 1, len(ps)):
                    trip.add((x, ps[i1], ps[i2]))
    vtl = np.array([(p, local[p][x], q, local[q][x]) for (x, p, q) in sorted(trip)], dtype=np.int64).reshape(-1, 4)
    return SplitGraph(n=n, subgraphs=out, vtl=vtl)
