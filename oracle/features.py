"""Eight local features of every line end, from the oracle's split — TEST INFRASTRUCTURE ONLY.

For end e at copy c (of vertex i, in subgraph j) on line t with twin copy c':
  0 log a_ii                  1 log a_ii^(c)  (the split weight of the copy, §4 step 3)
  2 log |O(i)| (copies of i)   3 number of lines at c (Fig. 7)
  4 log sum_{k != c} |Ã_j[c, k]|  (coupling inside the subgraph)
  5 log a_ii^(c')             6 log(max_k |a_ik| / min_k |a_ik|) over the neighbours of i in A
  7 log(n / n_j)
End order: 2t = side a, 2t + 1 = side b of line t (the split's line order).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .evs import SplitGraph, _as_csr


def line_features(split: SplitGraph, A, lines=None) -> np.ndarray:
    """Features of every end, rows in end order; with ``lines`` (indices into split.vtl) only the
    ends of those lines, rows 2k and 2k + 1 for the k-th listed line (the counts of copies and of
    lines at a copy still come from the whole split)."""
    A = _as_csr(A)
    m = len(split.vtl)
    ncopies = np.zeros(split.n, dtype=np.int64)
    for g in split.subgraphs:
        np.add.at(ncopies, g.vertices, 1)
    nlines = {}
    for (ja, ca, jb, cb) in split.vtl:
        nlines[(ja, ca)] = nlines.get((ja, ca), 0) + 1
        nlines[(jb, cb)] = nlines.get((jb, cb), 0) + 1
    diag = A.diagonal()
    sel = range(m) if lines is None else [int(t) for t in lines]
    out = np.zeros((2 * len(sel), 8))
    for k, t in enumerate(sel):
        ja, ca, jb, cb = split.vtl[t]
        for side, (j, c, jt, ct) in enumerate(((ja, ca, jb, cb), (jb, cb, ja, ca))):
            g = split.subgraphs[j]
            i = int(g.vertices[c])
            row = g.A.getrow(c).toarray().ravel()
            dc = row[c]
            off = np.abs(np.delete(row, c)).sum()
            dt = split.subgraphs[jt].A[ct, ct]
            nb = A.getrow(i)
            vals = np.abs(nb.data[nb.indices != i])
            f = out[2 * k + side]
            f[0] = np.log(diag[i])
            f[1] = np.log(dc)
            f[2] = np.log(ncopies[i])
            f[3] = nlines[(j, c)]
            f[4] = np.log(max(off, 1e-300))
            f[5] = np.log(dt)
            f[6] = np.log(vals.max() / vals.min()) if len(vals) else 0.0
            f[7] = np.log(split.n / len(g.vertices))
    return out
