// Electric Vertex Splitting (§4 steps 1-4, App. 2) — host implementation behind vtm_partition_evs.
//
// Split rule (the paper leaves the shares open, §4 "plenty of ways"): an edge (i,j) goes to every
// subgraph of O(i)∩O(j) with weight a_ij/|O(i)∩O(j)|; a boundary copy gets
// sum_{j!=i}|a_ij^(c)| + delta_i/|O(i)|, delta_i = a_ii - sum_{j!=i}|a_ij| (weak diagonal
// dominance keeps every piece SNND, Cor. 4.1); inner vertices keep a_ii; b_i is shared equally.
// Grid lines follow the hypercube of Fig. 7.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <thread>
#include <tuple>

#include "internal.h"

namespace {

using vtm::fail;

constexpr double kExcessTol = 64.0 * 2.220446049250313e-16;

double boundary_excess(double aii, double offabs) {
  double d = aii - offabs;
  if (d < 0) {
    if (d >= -kExcessTol * std::fabs(aii)) return 0.0;
    fail(VTM_ERR_NOT_CONFORMAL, "boundary vertex is not weakly diagonally dominant (delta_i < 0)");
  }
  return d;
}

template <class F>
void parallel_for(int64_t count, F&& f) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (count < 64 || nt == 1) {
    for (int64_t i = 0; i < count; ++i) f(i);
    return;
  }
  // any exception of a worker (an Error, or bad_alloc from a growing list) is carried back to
  // the calling thread and rethrown there, where the C ABI turns it into an error code
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> errs(nt);
  try {
    for (unsigned t = 0; t < nt; ++t) {
      th.emplace_back([&, t] {
        try {
          for (int64_t i = t; i < count; i += nt) f(i);
        } catch (...) {
          errs[t] = std::current_exception();
        }
      });
    }
  } catch (...) {  // a thread that could not start: wait for those that did, then report
    for (auto& x : th) x.join();
    throw;
  }
  for (auto& x : th) x.join();
  for (unsigned t = 0; t < nt; ++t)
    if (errs[t]) std::rethrow_exception(errs[t]);
}

void copy_and_check_matrix(const vtm_csr* A, vtm_partition* p) {
  if (!A || A->n <= 0 || !A->rowptr || !A->col || !A->val) fail(VTM_ERR_INVALID, "A: null or empty matrix");
  const int64_t n = A->n;
  if (A->nnz < 0 || A->rowptr[0] != 0 || A->rowptr[n] != A->nnz)
    fail(VTM_ERR_INVALID, "A: rowptr inconsistent with nnz");
  // every row's range first: a row's symmetric partner may lie in a later row, whose range must
  // already be known to lie inside [0, nnz]
  for (int64_t i = 0; i < n; ++i)
    if (A->rowptr[i + 1] < A->rowptr[i]) fail(VTM_ERR_INVALID, "A: rowptr not monotone");
  p->n = n;
  p->a_rowptr.assign(A->rowptr, A->rowptr + n + 1);
  p->a_col.assign(A->col, A->col + A->nnz);
  p->a_val.assign(A->val, A->val + A->nnz);
  // then the entries, blocks of consecutive rows on the host threads; each block keeps its first
  // error and the lowest block's is reported, so the error is the one a loop over the rows meets
  // first
  const int64_t kRows = 16384, nblk = (n + kRows - 1) / kRows;
  std::vector<int> ecode(nblk, 0);
  std::vector<std::string> emsg(nblk);
  parallel_for(nblk, [&](int64_t blk) {
    try {
      for (int64_t i = blk * kRows; i < std::min(n, (blk + 1) * kRows); ++i) {
        const int64_t lo = A->rowptr[i], hi = A->rowptr[i + 1];
        bool diag = false;
        for (int64_t k = lo; k < hi; ++k) {
          int32_t j = A->col[k];
          if (j < 0 || j >= n) fail(VTM_ERR_INVALID, "A: column index out of range");
          if (k > lo && A->col[k - 1] >= j) fail(VTM_ERR_INVALID, "A: columns not strictly ascending in a row");
          if (j == i) {
            diag = true;
            if (!(A->val[k] > 0)) fail(VTM_ERR_INVALID, "A: non-positive diagonal");
            continue;
          }
          // symmetric partner
          const int32_t* b = A->col + A->rowptr[j];
          const int32_t* e = A->col + A->rowptr[j + 1];
          const int32_t* f = std::lower_bound(b, e, (int32_t)i);
          if (f == e || *f != i || A->val[A->rowptr[j] + (f - b)] != A->val[k])
            fail(VTM_ERR_NOT_SYMMETRIC, "A is not symmetric");
        }
        if (!diag) fail(VTM_ERR_INVALID, "A: missing diagonal entry");
      }
    } catch (const vtm::Error& e) {
      ecode[blk] = e.code;
      emsg[blk] = e.msg;
    }
  });
  for (int64_t blk = 0; blk < nblk; ++blk)
    if (ecode[blk]) fail(ecode[blk], emsg[blk]);
}

// ----------------------------------------------------------------------------------- GRID

struct Axis {
  int m = 1, s = 1, nb = 1;
  // blocks containing coordinate c form the range [lo(c), hi(c)]
  // block q covers [q*s, min((q+1)*s, m-1)]; a cut coordinate c = q*s (q >= 1) is shared by
  // blocks q-1 and q when block q exists.
  int lo(int c) const {
    int q = c / s;
    return (c % s == 0 && c > 0) ? q - 1 : std::min(q, nb - 1);
  }
  int hi(int c) const {
    int q = c / s;
    if (c % s == 0 && c > 0) return q <= nb - 1 ? q : q - 1;
    return std::min(q, nb - 1);
  }
  int lo_of_block(int q) const { return q * s; }
  int hi_of_block(int q) const { return std::min((q + 1) * s, m - 1); }
};

void build_grid(const vtm_partition_spec* sp, vtm_partition* p) {
  Axis ax[3];
  int64_t nn = 1;
  for (int a = 0; a < 3; ++a) {
    int m = sp->dims[a], s = sp->block[a];
    if (m < 1 || s < 1) fail(VTM_ERR_INVALID, "grid: dims and block must be >= 1");
    ax[a].m = m;
    ax[a].s = s;
    ax[a].nb = (m > 1) ? (int)((m - 1 + s - 1) / s) : 1;
    if (ax[a].nb < 1) ax[a].nb = 1;
    nn *= m;
  }
  if (nn != p->n) fail(VTM_ERR_INVALID, "grid: dims do not match n");
  const int nx = ax[0].m, ny = ax[1].m;
  const int Bx = ax[0].nb, By = ax[1].nb, Bz = ax[2].nb;
  const int64_t np = (int64_t)Bx * By * Bz;
  if (np > INT32_MAX) fail(VTM_ERR_INVALID, "grid: too many blocks");
  p->npieces = (int32_t)np;
  // copies per piece
  p->piece_ptr.assign(np + 1, 0);
  std::vector<int> ext(np * 3), org(np * 3);
  for (int64_t j = 0; j < np; ++j) {
    int q[3] = {(int)(j % Bx), (int)((j / Bx) % By), (int)(j / ((int64_t)Bx * By))};
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      org[j * 3 + a] = ax[a].lo_of_block(q[a]);
      ext[j * 3 + a] = ax[a].hi_of_block(q[a]) - org[j * 3 + a] + 1;
      cnt *= ext[j * 3 + a];
    }
    p->piece_ptr[j + 1] = p->piece_ptr[j] + cnt;
  }
  const int64_t C = p->piece_ptr[np];
  p->copy_vertex.resize(C);
  p->copy_share.resize(C);
  auto nown = [&](int x, int y, int z) {
    return (int64_t)(ax[0].hi(x) - ax[0].lo(x) + 1) * (ax[1].hi(y) - ax[1].lo(y) + 1) * (ax[2].hi(z) - ax[2].lo(z) + 1);
  };
  auto common1 = [&](const Axis& A, int c, int d) {
    int lo = std::max(A.lo(c), A.lo(d)), hi = std::min(A.hi(c), A.hi(d));
    return hi >= lo ? hi - lo + 1 : 0;
  };
  // pass 1: row counts
  std::vector<int64_t> rowcnt(C + 1, 0);
  parallel_for(np, [&](int64_t j) {
    const int* o = &org[j * 3];
    const int* e = &ext[j * 3];
    int64_t c = p->piece_ptr[j];
    for (int z = 0; z < e[2]; ++z)
      for (int y = 0; y < e[1]; ++y)
        for (int x = 0; x < e[0]; ++x, ++c) {
          int gx = o[0] + x, gy = o[1] + y, gz = o[2] + z;
          int64_t v = gx + (int64_t)nx * (gy + (int64_t)ny * gz);
          p->copy_vertex[c] = v;
          p->copy_share[c] = 1.0 / (double)nown(gx, gy, gz);
          int64_t cnt = 0;
          for (int64_t k = p->a_rowptr[v]; k < p->a_rowptr[v + 1]; ++k) {
            int64_t u = p->a_col[k];
            if (u == v) { ++cnt; continue; }
            int ux = (int)(u % nx), uy = (int)((u / nx) % ny), uz = (int)(u / ((int64_t)nx * ny));
            if (ux >= o[0] && ux < o[0] + e[0] && uy >= o[1] && uy < o[1] + e[1] && uz >= o[2] && uz < o[2] + e[2]) ++cnt;
          }
          rowcnt[c + 1] = cnt;
        }
  });
  p->l_rowptr.resize(C + 1);
  p->l_rowptr[0] = 0;
  for (int64_t c = 0; c < C; ++c) p->l_rowptr[c + 1] = p->l_rowptr[c] + rowcnt[c + 1];
  p->l_col.resize(p->l_rowptr[C]);
  p->l_val.resize(p->l_rowptr[C]);
  // pass 2: values (step 3)
  parallel_for(np, [&](int64_t j) {
    const int* o = &org[j * 3];
    const int* e = &ext[j * 3];
    for (int64_t c = p->piece_ptr[j]; c < p->piece_ptr[j + 1]; ++c) {
      int64_t v = p->copy_vertex[c];
      int gx = (int)(v % nx), gy = (int)((v / nx) % ny), gz = (int)(v / ((int64_t)nx * ny));
      int64_t nv = nown(gx, gy, gz);
      int64_t pos = p->l_rowptr[c];
      int64_t diagpos = -1;
      double offabs = 0.0, inpiece = 0.0, aii = 0.0;
      for (int64_t k = p->a_rowptr[v]; k < p->a_rowptr[v + 1]; ++k) {
        int64_t u = p->a_col[k];
        double a = p->a_val[k];
        if (u == v) {
          aii = a;
          diagpos = pos;
          p->l_col[pos++] = (int32_t)(c - p->piece_ptr[j]);
          continue;
        }
        offabs += std::fabs(a);
        int ux = (int)(u % nx), uy = (int)((u / nx) % ny), uz = (int)(u / ((int64_t)nx * ny));
        int64_t cm = (int64_t)common1(ax[0], gx, ux) * common1(ax[1], gy, uy) * common1(ax[2], gz, uz);
        if (cm == 0) fail(VTM_ERR_INVALID, "grid: an edge of A lies in no common block");
        if (ux >= o[0] && ux < o[0] + e[0] && uy >= o[1] && uy < o[1] + e[1] && uz >= o[2] && uz < o[2] + e[2]) {
          double sh = a / (double)cm;
          int32_t lc = (ux - o[0]) + e[0] * ((uy - o[1]) + e[1] * (uz - o[2]));
          p->l_col[pos] = lc;
          p->l_val[pos++] = sh;
          inpiece += std::fabs(sh);
        }
      }
      if (nv == 1) p->l_val[diagpos] = aii;
      else p->l_val[diagpos] = inpiece + boundary_excess(aii, offabs) / (double)nv;
    }
  });
  // step 4: hypercube lines; and boundary count
  int64_t nbnd = 0;
  auto copy_id = [&](int qx, int qy, int qz, int gx, int gy, int gz) {
    int64_t j = qx + (int64_t)Bx * (qy + (int64_t)By * qz);
    const int* o = &org[j * 3];
    const int* e = &ext[j * 3];
    return p->piece_ptr[j] + (gx - o[0]) + (int64_t)e[0] * ((gy - o[1]) + (int64_t)e[1] * (gz - o[2]));
  };
  for (int gz = 0; gz < ax[2].m; ++gz)
    for (int gy = 0; gy < ax[1].m; ++gy)
      for (int gx = 0; gx < ax[0].m; ++gx) {
        int lo[3] = {ax[0].lo(gx), ax[1].lo(gy), ax[2].lo(gz)};
        int hi[3] = {ax[0].hi(gx), ax[1].hi(gy), ax[2].hi(gz)};
        if (lo[0] == hi[0] && lo[1] == hi[1] && lo[2] == hi[2]) continue;
        ++nbnd;
        for (int a = 0; a < 3; ++a) {
          if (lo[a] == hi[a]) continue;
          int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
          for (int q1 = lo[b1]; q1 <= hi[b1]; ++q1)
            for (int q2 = lo[b2]; q2 <= hi[b2]; ++q2) {
              int qa[3], qb[3];
              qa[a] = lo[a];
              qb[a] = hi[a];
              qa[b1] = qb[b1] = q1;
              qa[b2] = qb[b2] = q2;
              p->line_a.push_back(copy_id(qa[0], qa[1], qa[2], gx, gy, gz));
              p->line_b.push_back(copy_id(qb[0], qb[1], qb[2], gx, gy, gz));
            }
        }
      }
  p->nboundary = nbnd;
}

// ----------------------------------------------------------------------------------- OWNERS

void build_owners(const vtm_partition_spec* sp, vtm_partition* p) {
  const int64_t n = p->n;
  const int32_t np = sp->npieces;
  if (np < 1 || !sp->owner_ptr || !sp->owner_piece) fail(VTM_ERR_INVALID, "owners: missing owner sets");
  if (sp->owner_ptr[0] != 0) fail(VTM_ERR_INVALID, "owners: owner_ptr[0] != 0");
  p->npieces = np;
  std::vector<std::vector<int64_t>> verts(np);
  int64_t nbnd = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t lo = sp->owner_ptr[i], hi = sp->owner_ptr[i + 1];
    if (hi <= lo) fail(VTM_ERR_INVALID, "owners: a vertex has no owner");
    if (hi - lo > 1) ++nbnd;
    for (int64_t k = lo; k < hi; ++k) {
      int32_t q = sp->owner_piece[k];
      if (q < 0 || q >= np || (k > lo && sp->owner_piece[k - 1] >= q)) fail(VTM_ERR_INVALID, "owners: bad or unsorted owner list");
      verts[q].push_back(i);
    }
  }
  p->nboundary = nbnd;
  p->piece_ptr.assign(np + 1, 0);
  for (int32_t q = 0; q < np; ++q) p->piece_ptr[q + 1] = p->piece_ptr[q] + (int64_t)verts[q].size();
  const int64_t C = p->piece_ptr[np];
  p->copy_vertex.resize(C);
  p->copy_share.resize(C);
  auto owners = [&](int64_t i) { return std::make_pair(sp->owner_piece + sp->owner_ptr[i], sp->owner_piece + sp->owner_ptr[i + 1]); };
  auto local_of = [&](int32_t q, int64_t v) -> int64_t {
    auto& vs = verts[q];
    auto it = std::lower_bound(vs.begin(), vs.end(), v);
    if (it == vs.end() || *it != v) return -1;
    return it - vs.begin();
  };
  auto ncommon = [&](int64_t i, int64_t j) {
    auto a = owners(i), b = owners(j);
    int64_t c = 0;
    const int32_t *x = a.first, *y = b.first;
    while (x < a.second && y < b.second) {
      if (*x == *y) { ++c; ++x; ++y; }
      else if (*x < *y) ++x;
      else ++y;
    }
    return c;
  };
  std::vector<int64_t> rowcnt(C + 1, 0);
  for (int32_t q = 0; q < np; ++q)
    for (size_t l = 0; l < verts[q].size(); ++l) {
      int64_t c = p->piece_ptr[q] + (int64_t)l, v = verts[q][l];
      p->copy_vertex[c] = v;
      p->copy_share[c] = 1.0 / (double)(sp->owner_ptr[v + 1] - sp->owner_ptr[v]);
      int64_t cnt = 0;
      for (int64_t k = p->a_rowptr[v]; k < p->a_rowptr[v + 1]; ++k)
        if (p->a_col[k] == v || local_of(q, p->a_col[k]) >= 0) ++cnt;
      rowcnt[c + 1] = cnt;
    }
  p->l_rowptr.resize(C + 1);
  p->l_rowptr[0] = 0;
  for (int64_t c = 0; c < C; ++c) p->l_rowptr[c + 1] = p->l_rowptr[c] + rowcnt[c + 1];
  p->l_col.resize(p->l_rowptr[C]);
  p->l_val.resize(p->l_rowptr[C]);
  for (int32_t q = 0; q < np; ++q)
    for (size_t l = 0; l < verts[q].size(); ++l) {
      int64_t c = p->piece_ptr[q] + (int64_t)l, v = verts[q][l];
      int64_t nv = sp->owner_ptr[v + 1] - sp->owner_ptr[v];
      int64_t pos = p->l_rowptr[c], diagpos = -1;
      double offabs = 0, inpiece = 0, aii = 0;
      for (int64_t k = p->a_rowptr[v]; k < p->a_rowptr[v + 1]; ++k) {
        int64_t u = p->a_col[k];
        double a = p->a_val[k];
        if (u == v) {
          aii = a;
          diagpos = pos;
          p->l_col[pos++] = (int32_t)l;
          continue;
        }
        offabs += std::fabs(a);
        int64_t cm = ncommon(v, u);
        if (cm == 0) fail(VTM_ERR_INVALID, "owners: an edge of A lies in no common subgraph");
        int64_t lu = local_of(q, u);
        if (lu >= 0) {
          double sh = a / (double)cm;
          p->l_col[pos] = (int32_t)lu;
          p->l_val[pos++] = sh;
          inpiece += std::fabs(sh);
        }
      }
      p->l_val[diagpos] = (nv == 1) ? aii : inpiece + boundary_excess(aii, offabs) / (double)nv;
    }
  for (int64_t t = 0; t < sp->nlines; ++t) {
    int64_t v = sp->line_vertex[t];
    if (v < 0 || v >= n) fail(VTM_ERR_INVALID, "owners: line vertex out of range");
    int32_t qa = sp->line_piece_a[t], qb = sp->line_piece_b[t];
    if (qa < 0 || qa >= np || qb < 0 || qb >= np || qa == qb) fail(VTM_ERR_INVALID, "owners: bad line pieces");
    int64_t la = local_of(qa, v), lb = local_of(qb, v);
    if (la < 0 || lb < 0) fail(VTM_ERR_INVALID, "owners: line joins a copy that does not exist");
    p->line_a.push_back(p->piece_ptr[qa] + la);
    p->line_b.push_back(p->piece_ptr[qb] + lb);
  }
}

// ----------------------------------------------------------------------------------- EXPLICIT

void build_explicit(const vtm_partition_spec* sp, vtm_partition* p) {
  const int32_t np = sp->npieces;
  if (np < 1 || !sp->piece_ptr || !sp->copy_vertex || !sp->copy_share || !sp->local_rowptr || !sp->local_col || !sp->local_val)
    fail(VTM_ERR_INVALID, "explicit: missing arrays");
  p->npieces = np;
  p->piece_ptr.assign(sp->piece_ptr, sp->piece_ptr + np + 1);
  if (p->piece_ptr[0] != 0) fail(VTM_ERR_INVALID, "explicit: piece_ptr[0] != 0");
  for (int32_t q = 0; q < np; ++q)
    if (p->piece_ptr[q + 1] < p->piece_ptr[q]) fail(VTM_ERR_INVALID, "explicit: piece_ptr not monotone");
  const int64_t C = p->piece_ptr[np];
  p->copy_vertex.assign(sp->copy_vertex, sp->copy_vertex + C);
  p->copy_share.assign(sp->copy_share, sp->copy_share + C);
  p->l_rowptr.assign(sp->local_rowptr, sp->local_rowptr + C + 1);
  if (p->l_rowptr[0] != 0) fail(VTM_ERR_INVALID, "explicit: local_rowptr[0] != 0");
  const int64_t nnz = p->l_rowptr[C];
  p->l_col.assign(sp->local_col, sp->local_col + nnz);
  p->l_val.assign(sp->local_val, sp->local_val + nnz);
  std::vector<int64_t> cnt(p->n, 0);
  for (int32_t q = 0; q < np; ++q) {
    int64_t nq = p->piece_ptr[q + 1] - p->piece_ptr[q];
    for (int64_t c = p->piece_ptr[q]; c < p->piece_ptr[q + 1]; ++c) {
      if (p->copy_vertex[c] < 0 || p->copy_vertex[c] >= p->n) fail(VTM_ERR_INVALID, "explicit: copy vertex out of range");
      cnt[p->copy_vertex[c]]++;
      for (int64_t k = p->l_rowptr[c]; k < p->l_rowptr[c + 1]; ++k)
        if (p->l_col[k] < 0 || p->l_col[k] >= nq) fail(VTM_ERR_INVALID, "explicit: local column out of range");
    }
  }
  int64_t nbnd = 0;
  for (int64_t i = 0; i < p->n; ++i) {
    if (cnt[i] == 0) fail(VTM_ERR_INVALID, "explicit: a vertex has no copy");
    if (cnt[i] > 1) ++nbnd;
  }
  p->nboundary = nbnd;
  for (int64_t t = 0; t < sp->ncopy_lines; ++t) {
    int64_t a = sp->line_copy_a[t], b = sp->line_copy_b[t];
    if (a < 0 || a >= C || b < 0 || b >= C || a == b || p->copy_vertex[a] != p->copy_vertex[b])
      fail(VTM_ERR_INVALID, "explicit: a line must join two copies of the same vertex");
    p->line_a.push_back(a);
    p->line_b.push_back(b);
  }
}

}  // namespace

namespace vtm {
void build_elements(const vtm_partition_spec* sp, vtm_partition* p);
void build_conformal(const vtm_partition_spec* sp, vtm_partition* p);
void build_partition(const vtm_csr* A, const vtm_partition_spec* spec, vtm_partition* p) {
  if (!spec) fail(VTM_ERR_INVALID, "null partition spec");
  copy_and_check_matrix(A, p);
  switch (spec->kind) {
    case VTM_PART_GRID: build_grid(spec, p); break;
    case VTM_PART_OWNERS: build_owners(spec, p); break;
    case VTM_PART_EXPLICIT: build_explicit(spec, p); break;
    case VTM_PART_ELEMENTS: build_elements(spec, p); break;
    case VTM_PART_CONFORMAL: build_conformal(spec, p); break;
    default: fail(VTM_ERR_INVALID, "unknown partition kind");
  }
  // every copy that has a line must sit in a piece; pieces must be non-empty
  for (int32_t q = 0; q < p->npieces; ++q)
    if (p->piece_ptr[q + 1] == p->piece_ptr[q]) fail(VTM_ERR_INVALID, "a subgraph is empty");
}
}  // namespace vtm

namespace vtm {

// Candidate couplings of §7.2 (vtm_partition_line_pairs): pairs t < u of lines joining the same
// two subgraphs whose copies are neighbours on both sides, with |a_ik| of the original matrix.
void line_pairs(const vtm_partition* p, std::vector<int64_t>& pairs, std::vector<double>& wts) {
  pairs.clear();
  wts.clear();
  const int64_t nl = (int64_t)p->line_a.size();
  const int64_t C = p->piece_ptr[p->npieces];
  std::vector<int32_t> piece(C);
  for (int32_t j = 0; j < p->npieces; ++j)
    for (int64_t c = p->piece_ptr[j]; c < p->piece_ptr[j + 1]; ++c) piece[c] = j;
  // lines at each copy
  std::vector<int64_t> lptr(C + 1, 0), lid(2 * nl);
  for (int64_t t = 0; t < nl; ++t) {
    lptr[p->line_a[t] + 1]++;
    lptr[p->line_b[t] + 1]++;
  }
  for (int64_t c = 0; c < C; ++c) lptr[c + 1] += lptr[c];
  {
    std::vector<int64_t> fill(lptr.begin(), lptr.end() - 1);
    for (int64_t t = 0; t < nl; ++t) {
      lid[fill[p->line_a[t]]++] = t;
      lid[fill[p->line_b[t]]++] = t;
    }
  }
  auto has_col = [&](int64_t c, int64_t lc) {
    for (int64_t k = p->l_rowptr[c]; k < p->l_rowptr[c + 1]; ++k)
      if (p->l_col[k] == lc) return true;
    return false;
  };
  auto a_abs = [&](int64_t i, int64_t k) {
    for (int64_t q = p->a_rowptr[i]; q < p->a_rowptr[i + 1]; ++q)
      if (p->a_col[q] == k) return std::fabs(p->a_val[q]);
    return 0.0;
  };
  // blocks of consecutive lines on the host threads, each into its own lists; joined in block
  // order, so the pairs come out in the same order as from one loop over t
  const int64_t kBlock = 4096, nblk = (nl + kBlock - 1) / kBlock;
  std::vector<std::vector<int64_t>> bpairs(nblk);
  std::vector<std::vector<double>> bwts(nblk);
  parallel_for(nblk, [&](int64_t blk) {
    std::vector<int64_t>& pp = bpairs[blk];
    std::vector<double>& ww = bwts[blk];
    for (int64_t t = blk * kBlock; t < std::min(nl, (blk + 1) * kBlock); ++t) {
      const int64_t ca = p->line_a[t], cb = p->line_b[t];
      const int32_t ja = piece[ca], jb = piece[cb];
      for (int64_t k = p->l_rowptr[ca]; k < p->l_rowptr[ca + 1]; ++k) {
        const int64_t cn = p->piece_ptr[ja] + p->l_col[k];
        if (cn == ca) continue;
        for (int64_t q = lptr[cn]; q < lptr[cn + 1]; ++q) {
          const int64_t u = lid[q];
          if (u <= t) continue;
          const int64_t ua = p->line_a[u], ub = p->line_b[u];
          int64_t other;  // u's copy in jb
          if (piece[ua] == ja && piece[ub] == jb) other = ub;
          else if (piece[ub] == ja && piece[ua] == jb) other = ua;
          else continue;
          if (!has_col(cb, other - p->piece_ptr[jb])) continue;
          pp.push_back(t);
          pp.push_back(u);
          ww.push_back(a_abs(p->copy_vertex[ca], p->copy_vertex[cn]));
        }
      }
    }
  });
  size_t total = 0;
  for (const auto& v : bwts) total += v.size();
  pairs.reserve(2 * total);
  wts.reserve(total);
  for (int64_t blk = 0; blk < nblk; ++blk) {
    pairs.insert(pairs.end(), bpairs[blk].begin(), bpairs[blk].end());
    wts.insert(wts.end(), bwts[blk].begin(), bwts[blk].end());
  }
}

// Eight local features of every line end (see vtm_line_features in vtm.h), in API end order.
void line_features(const vtm_partition* p, float* out) {
  const int64_t C = p->piece_ptr[p->npieces];
  const int64_t nl = (int64_t)p->line_a.size();
  std::vector<int32_t> ncopies(p->n, 0), nlines(C, 0), piece(C, 0);
  for (int64_t c = 0; c < C; ++c) ncopies[p->copy_vertex[c]]++;
  for (int64_t t = 0; t < nl; ++t) {
    nlines[p->line_a[t]]++;
    nlines[p->line_b[t]]++;
  }
  for (int32_t j = 0; j < p->npieces; ++j)
    for (int64_t c = p->piece_ptr[j]; c < p->piece_ptr[j + 1]; ++c) piece[c] = j;
  auto safe_log = [](double v) { return std::log(std::max(v, 1e-300)); };
  auto copy_diag_and_off = [&](int64_t c, double* d, double* off) {
    const int64_t l = c - p->piece_ptr[piece[c]];
    *d = 0;
    *off = 0;
    for (int64_t k = p->l_rowptr[c]; k < p->l_rowptr[c + 1]; ++k) {
      if (p->l_col[k] == l) *d += p->l_val[k];
      else *off += std::fabs(p->l_val[k]);
    }
  };
  // every end writes its own row: blocks of consecutive ends on the host threads
  const int64_t E = 2 * nl, kBlock = 4096;
  parallel_for((E + kBlock - 1) / kBlock, [&](int64_t blk) {
    for (int64_t e = blk * kBlock; e < std::min(E, (blk + 1) * kBlock); ++e) {
      const int64_t c = (e & 1) ? p->line_b[e >> 1] : p->line_a[e >> 1];
      const int64_t tw = (e & 1) ? p->line_a[e >> 1] : p->line_b[e >> 1];
      const int64_t i = p->copy_vertex[c];
      double aii = 0, amax = 0, amin = INFINITY;
      for (int64_t k = p->a_rowptr[i]; k < p->a_rowptr[i + 1]; ++k) {
        if (p->a_col[k] == i) aii = p->a_val[k];
        else {
          amax = std::max(amax, std::fabs(p->a_val[k]));
          amin = std::min(amin, std::fabs(p->a_val[k]));
        }
      }
      double dc, offc, dt, offt;
      copy_diag_and_off(c, &dc, &offc);
      copy_diag_and_off(tw, &dt, &offt);
      const int64_t nj = p->piece_ptr[piece[c] + 1] - p->piece_ptr[piece[c]];
      float* f = out + e * VTM_MLP_IN;
      f[0] = (float)safe_log(aii);
      f[1] = (float)safe_log(dc);
      f[2] = (float)std::log((double)ncopies[i]);
      f[3] = (float)nlines[c];
      f[4] = (float)safe_log(offc);
      f[5] = (float)safe_log(dt);
      f[6] = (amax > 0 && std::isfinite(amin) && amin > 0) ? (float)std::log(amax / amin) : 0.f;
      f[7] = (float)std::log((double)p->n / (double)nj);
    }
  });
}

}  // namespace vtm

// ------------------------------------------------------------------------------------------ ELEMENTS

namespace {

using vtm::fail;

void rcb(const double* coords, int dim, std::vector<int64_t>& ids, int64_t lo, int64_t hi, int32_t nparts, int32_t base,
         std::vector<int32_t>& piece) {
  if (nparts <= 1) {
    for (int64_t k = lo; k < hi; ++k) piece[ids[k]] = base;
    return;
  }
  const int32_t pl = nparts / 2;
  int axis = 0;
  double best = -1.0;
  for (int a = 0; a < dim; ++a) {
    double mn = INFINITY, mx = -INFINITY;
    for (int64_t k = lo; k < hi; ++k) {
      const double v = coords[ids[k] * dim + a];
      mn = std::min(mn, v);
      mx = std::max(mx, v);
    }
    if (mx - mn > best) {
      best = mx - mn;
      axis = a;
    }
  }
  std::sort(ids.begin() + lo, ids.begin() + hi, [&](int64_t x, int64_t y) {
    const double vx = coords[x * dim + axis], vy = coords[y * dim + axis];
    return vx < vy || (vx == vy && x < y);
  });
  const int64_t m = lo + ((hi - lo) * (int64_t)pl) / nparts;
  rcb(coords, dim, ids, lo, m, pl, base, piece);
  rcb(coords, dim, ids, m, hi, nparts - pl, base + pl, piece);
}

// Reverse Cuthill-McKee order of a small graph given as adjacency lists over 0..m-1.
std::vector<int32_t> rcm_order(const std::vector<std::vector<int32_t>>& adj) {
  const int32_t m = (int32_t)adj.size();
  std::vector<int32_t> order;
  order.reserve(m);
  std::vector<char> seen(m, 0);
  auto deg = [&](int32_t v) { return (int32_t)adj[v].size(); };
  for (;;) {
    int32_t start = -1;
    for (int32_t v = 0; v < m; ++v)
      if (!seen[v] && (start < 0 || deg(v) < deg(start))) start = v;
    if (start < 0) break;
    const size_t first = order.size();
    order.push_back(start);
    seen[start] = 1;
    for (size_t h = first; h < order.size(); ++h) {
      std::vector<int32_t> nb;
      for (int32_t u : adj[order[h]])
        if (!seen[u]) {
          seen[u] = 1;
          nb.push_back(u);
        }
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) { return deg(a) < deg(b) || (deg(a) == deg(b) && a < b); });
      for (int32_t u : nb) order.push_back(u);
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

}  // namespace

namespace vtm {

void build_elements(const vtm_partition_spec* sp, vtm_partition* p) {
  const int64_t ne = sp->nelem;
  const int k = sp->nodes_per_elem;
  if (ne < 1 || k < 2 || k > 64 || !sp->elem_nodes || !sp->elem_mats || !sp->node_unknown || sp->nnodes < 1)
    fail(VTM_ERR_INVALID, "elements: missing arrays");
  if (sp->npieces < 1) fail(VTM_ERR_INVALID, "elements: npieces must be >= 1");
  const int32_t np = sp->npieces;
  p->npieces = np;
  std::vector<int32_t> epiece(ne);
  if (sp->elem_piece) {
    for (int64_t e = 0; e < ne; ++e) {
      epiece[e] = sp->elem_piece[e];
      if (epiece[e] < 0 || epiece[e] >= np) fail(VTM_ERR_INVALID, "elements: piece id out of range");
    }
  } else {
    if (!sp->elem_coords || sp->coord_dim < 1 || sp->coord_dim > 3) fail(VTM_ERR_INVALID, "elements: RCB needs coordinates");
    if (np > ne) fail(VTM_ERR_INVALID, "elements: more pieces than elements");
    std::vector<int64_t> ids(ne);
    for (int64_t e = 0; e < ne; ++e) ids[e] = e;
    rcb(sp->elem_coords, sp->coord_dim, ids, 0, ne, np, 0, epiece);
  }
  auto unk = [&](int64_t node) -> int64_t {
    if (node < 0 || node >= sp->nnodes) fail(VTM_ERR_INVALID, "elements: node id out of range");
    const int64_t u = sp->node_unknown[node];
    if (u >= p->n) fail(VTM_ERR_INVALID, "elements: unknown index out of range");
    return u;
  };
  // elements of each piece
  std::vector<std::vector<int64_t>> pel(np);
  for (int64_t e = 0; e < ne; ++e) pel[epiece[e]].push_back(e);
  // per piece: vertices (unknowns), RCM order, local matrix
  std::vector<std::vector<int64_t>> pverts(np);
  std::vector<std::vector<int64_t>> prow_cols(np);
  std::vector<int64_t> ncop(p->n, 0);
  struct Local {
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
    std::vector<double> val;
  };
  std::vector<Local> loc(np);
  parallel_for(np, [&](int64_t jj) {
    const int32_t j = (int32_t)jj;
    std::vector<int64_t> vs;
    for (int64_t e : pel[j])
      for (int a = 0; a < k; ++a) {
        const int64_t u = unk(sp->elem_nodes[e * k + a]);
        if (u >= 0) vs.push_back(u);
      }
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    const int32_t m = (int32_t)vs.size();
    auto lid = [&](int64_t u) { return (int32_t)(std::lower_bound(vs.begin(), vs.end(), u) - vs.begin()); };
    std::vector<std::vector<int32_t>> adj(m);
    for (int64_t e : pel[j])
      for (int a = 0; a < k; ++a) {
        const int64_t ua = unk(sp->elem_nodes[e * k + a]);
        if (ua < 0) continue;
        for (int b = 0; b < k; ++b) {
          const int64_t ub = unk(sp->elem_nodes[e * k + b]);
          if (ub < 0 || b == a) continue;
          adj[lid(ua)].push_back(lid(ub));
        }
      }
    for (auto& l : adj) {
      std::sort(l.begin(), l.end());
      l.erase(std::unique(l.begin(), l.end()), l.end());
    }
    const std::vector<int32_t> ord = rcm_order(adj);  // ord[new] = old
    std::vector<int32_t> newid(m);
    for (int32_t t = 0; t < m; ++t) newid[ord[t]] = t;
    // local matrix rows in the new order: sum of element contributions, columns merged
    std::vector<std::vector<std::pair<int32_t, double>>> rows(m);
    for (int64_t e : pel[j]) {
      const double* K = sp->elem_mats + e * k * k;
      for (int a = 0; a < k; ++a) {
        const int64_t ua = unk(sp->elem_nodes[e * k + a]);
        if (ua < 0) continue;
        const int32_t ra = newid[lid(ua)];
        for (int b = 0; b < k; ++b) {
          const int64_t ub = unk(sp->elem_nodes[e * k + b]);
          if (ub < 0) continue;
          rows[ra].emplace_back(newid[lid(ub)], K[a * k + b]);
        }
      }
    }
    Local& L = loc[j];
    L.rowptr.assign(m + 1, 0);
    for (int32_t r = 0; r < m; ++r) {
      auto& rr = rows[r];
      std::stable_sort(rr.begin(), rr.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (size_t q = 0; q < rr.size();) {
        size_t q2 = q;
        double v = 0.0;
        while (q2 < rr.size() && rr[q2].first == rr[q].first) v += rr[q2++].second;
        L.col.push_back(rr[q].first);
        L.val.push_back(v);
        q = q2;
      }
      L.rowptr[r + 1] = (int64_t)L.col.size();
    }
    std::vector<int64_t> vnew(m);
    for (int32_t t = 0; t < m; ++t) vnew[t] = vs[ord[t]];
    pverts[j] = std::move(vnew);
  });
  p->piece_ptr.assign(np + 1, 0);
  for (int32_t j = 0; j < np; ++j) {
    if (pverts[j].empty()) fail(VTM_ERR_INVALID, "elements: a subgraph has no unknowns");
    p->piece_ptr[j + 1] = p->piece_ptr[j] + (int64_t)pverts[j].size();
    for (int64_t u : pverts[j]) ncop[u]++;
  }
  for (int64_t i = 0; i < p->n; ++i)
    if (ncop[i] == 0) fail(VTM_ERR_INVALID, "elements: an unknown belongs to no element");
  const int64_t C = p->piece_ptr[np];
  p->copy_vertex.resize(C);
  p->copy_share.resize(C);
  p->l_rowptr.assign(C + 1, 0);
  int64_t nb = 0;
  for (int64_t i = 0; i < p->n; ++i) nb += ncop[i] > 1;
  p->nboundary = nb;
  for (int32_t j = 0; j < np; ++j) {
    const int64_t c0 = p->piece_ptr[j];
    const Local& L = loc[j];
    const int64_t k0 = (int64_t)p->l_col.size();
    for (size_t t = 0; t < pverts[j].size(); ++t) {
      p->copy_vertex[c0 + t] = pverts[j][t];
      p->copy_share[c0 + t] = 1.0 / (double)ncop[pverts[j][t]];
      p->l_rowptr[c0 + t + 1] = k0 + L.rowptr[t + 1];
    }
    p->l_col.insert(p->l_col.end(), L.col.begin(), L.col.end());
    p->l_val.insert(p->l_val.end(), L.val.begin(), L.val.end());
  }
  // lines: element edges through a vertex with elements of two subgraphs around them
  std::vector<std::tuple<int64_t, int64_t, int32_t>> edges;  // (lo node, hi node, piece)
  edges.reserve((size_t)ne * k * (k - 1) / 2);
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b) {
        const int64_t u = sp->elem_nodes[e * k + a], v = sp->elem_nodes[e * k + b];
        edges.emplace_back(std::min(u, v), std::max(u, v), epiece[e]);
      }
  std::sort(edges.begin(), edges.end());
  std::vector<std::tuple<int64_t, int32_t, int32_t>> trip;  // (vertex, pa, pb)
  for (size_t q = 0; q < edges.size();) {
    size_t q2 = q;
    std::vector<int32_t> ps;
    while (q2 < edges.size() && std::get<0>(edges[q2]) == std::get<0>(edges[q]) &&
           std::get<1>(edges[q2]) == std::get<1>(edges[q])) {
      ps.push_back(std::get<2>(edges[q2]));
      ++q2;
    }
    std::sort(ps.begin(), ps.end());
    ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
    if (ps.size() > 1)
      for (int64_t node : {std::get<0>(edges[q]), std::get<1>(edges[q])}) {
        const int64_t u = unk(node);
        if (u < 0) continue;
        for (size_t x = 0; x < ps.size(); ++x)
          for (size_t y = x + 1; y < ps.size(); ++y) trip.emplace_back(u, ps[x], ps[y]);
      }
    q = q2;
  }
  std::sort(trip.begin(), trip.end());
  trip.erase(std::unique(trip.begin(), trip.end()), trip.end());
  auto copy_of = [&](int32_t j, int64_t u) -> int64_t {
    const auto& vs = pverts[j];
    for (size_t t = 0; t < vs.size(); ++t)
      if (vs[t] == u) return p->piece_ptr[j] + (int64_t)t;
    fail(VTM_ERR_INVALID, "elements: line joins a missing copy");
  };
  // vertex -> (piece, copy) lookup through a per-piece hash would be faster; pieces are small
  std::vector<std::vector<std::pair<int64_t, int32_t>>> pindex(np);
  for (int32_t j = 0; j < np; ++j) {
    pindex[j].reserve(pverts[j].size());
    for (size_t t = 0; t < pverts[j].size(); ++t) pindex[j].emplace_back(pverts[j][t], (int32_t)t);
    std::sort(pindex[j].begin(), pindex[j].end());
  }
  auto copy_fast = [&](int32_t j, int64_t u) -> int64_t {
    const auto& ix = pindex[j];
    auto it = std::lower_bound(ix.begin(), ix.end(), std::make_pair(u, (int32_t)-1));
    if (it == ix.end() || it->first != u) return copy_of(j, u);
    return p->piece_ptr[j] + it->second;
  };
  for (const auto& t : trip) {
    p->line_a.push_back(copy_fast(std::get<1>(t), std::get<0>(t)));
    p->line_b.push_back(copy_fast(std::get<2>(t), std::get<0>(t)));
  }
}

void element_pieces(const vtm_partition_spec* sp, int32_t* out) {
  std::vector<int32_t> ep(sp->nelem);
  std::vector<int64_t> ids(sp->nelem);
  for (int64_t e = 0; e < sp->nelem; ++e) ids[e] = e;
  rcb(sp->elem_coords, sp->coord_dim, ids, 0, sp->nelem, sp->npieces, 0, ep);
  std::copy(ep.begin(), ep.end(), out);
}

}  // namespace vtm
