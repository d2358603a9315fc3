// VTM_PART_CONFORMAL: the general conformal split of App. 1 (Lemma A1.1, Thm 4.2) for SPD matrices
// that the diagonal rule of §4 step 3 cannot split (host only).
//
// One split of a subgraph with SPD matrix M over its copies: alpha = copies whose home is below the
// middle of the subgraph's id range, beta = the others; the boundary B = the alpha copies that M joins
// to a beta copy (so the interiors I_a = alpha \ B and I_b = beta are not joined).  Completing the
// square over each interior gives T_a = M_Ba M_aa^{-1} M_aB, T_b = M_Bb M_bb^{-1} M_bB and the Schur
// complement S = M_BB - T_a - T_b (SPD); the boundary copies are split so that the alpha subgraph gets
// T_a + lam S on B and the beta subgraph T_b + (1 - lam) S on new copies of B (both SPD, summing to
// M).  A new beta copy's home is the smallest home among its beta neighbours; its source share is
// (1 - lam) of the copy's, the alpha copy keeps lam; one line joins the two.  Repeated over the id
// halves until every subgraph holds one id (Thm 4.2: N - 1 splits).  Dense arithmetic: the boundary
// blocks fill in, and the interior solves use a dense Cholesky factor, O(n^3) work and O(n^2) memory.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"

namespace vtm {

namespace {

struct Dense {
  int n = 0;
  std::vector<double> a;  // row-major n x n
  double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * n + j]; }
};

// In-place lower Cholesky factor of an SPD matrix (row-major); false on a non-positive pivot.
bool cholesky(std::vector<double>& L, int n) {
  for (int j = 0; j < n; ++j) {
    double d = L[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double v = L[(size_t)i * n + j];
      const double* li = &L[(size_t)i * n];
      const double* lj = &L[(size_t)j * n];
      for (int k = 0; k < j; ++k) v -= li[k] * lj[k];
      L[(size_t)i * n + j] = v / ljj;
    }
  }
  return true;
}

// T = X^T M_ii^{-1} X for the block X = M[I, B] (|I| x |B|): with L L^T = M_ii, Y = L^{-1} X and
// T = Y^T Y.
std::vector<double> schur_term(const Dense& M, const std::vector<int>& I, const std::vector<int>& B) {
  const int ni = (int)I.size(), nb = (int)B.size();
  std::vector<double> T((size_t)nb * nb, 0.0);
  if (ni == 0 || nb == 0) return T;
  std::vector<double> L((size_t)ni * ni);
  for (int r = 0; r < ni; ++r)
    for (int c = 0; c < ni; ++c) L[(size_t)r * ni + c] = M(I[r], I[c]);
  if (!cholesky(L, ni)) fail(VTM_ERR_NOT_SPD, "conformal split: an interior block is not positive definite");
  // Y (ni x nb, row-major) = L^{-1} X by forward substitution, all columns at once
  std::vector<double> Y((size_t)ni * nb);
  for (int r = 0; r < ni; ++r)
    for (int c = 0; c < nb; ++c) Y[(size_t)r * nb + c] = M(I[r], B[c]);
  for (int r = 0; r < ni; ++r) {
    double* yr = &Y[(size_t)r * nb];
    for (int k = 0; k < r; ++k) {
      const double l = L[(size_t)r * ni + k];
      if (l == 0.0) continue;
      const double* yk = &Y[(size_t)k * nb];
      for (int c = 0; c < nb; ++c) yr[c] -= l * yk[c];
    }
    const double inv = 1.0 / L[(size_t)r * ni + r];
    for (int c = 0; c < nb; ++c) yr[c] *= inv;
  }
  for (int r = 0; r < ni; ++r) {
    const double* yr = &Y[(size_t)r * nb];
    for (int c1 = 0; c1 < nb; ++c1) {
      const double v = yr[c1];
      if (v == 0.0) continue;
      double* t = &T[(size_t)c1 * nb];
      for (int c2 = 0; c2 < nb; ++c2) t[c2] += v * yr[c2];
    }
  }
  return T;
}

struct Builder {
  double lam;
  std::vector<int64_t> cvert;   // parent vertex of each copy
  std::vector<int32_t> chome;
  std::vector<double> cshare;
  std::vector<std::pair<int64_t, int64_t>> lines;
  std::vector<std::vector<int64_t>> piece_ids;
  std::vector<Dense> piece_mat;

  void rec(std::vector<int64_t> ids, Dense M, int lo, int hi) {
    if (hi - lo == 1) {
      piece_ids[lo] = std::move(ids);
      piece_mat[lo] = std::move(M);
      return;
    }
    const int mid = (lo + hi) / 2;
    const int m = (int)ids.size();
    std::vector<int> a_side, b_side;
    for (int k = 0; k < m; ++k) (chome[ids[k]] < mid ? a_side : b_side).push_back(k);
    std::vector<int> B, Ia;
    for (int k : a_side) {
      bool bnd = false;
      for (int q : b_side)
        if (M(k, q) != 0.0) {
          bnd = true;
          break;
        }
      (bnd ? B : Ia).push_back(k);
    }
    const std::vector<int>& Ib = b_side;
    const int nb = (int)B.size();
    std::vector<double> Ta = schur_term(M, Ia, B), Tb = schur_term(M, Ib, B);
    std::vector<double> Sa((size_t)nb * nb), Sb((size_t)nb * nb);
    for (int r = 0; r < nb; ++r)
      for (int c = 0; c < nb; ++c) {
        const size_t k = (size_t)r * nb + c;
        const double S = M(B[r], B[c]) - Ta[k] - Tb[k];
        Sa[k] = Ta[k] + lam * S;
        Sb[k] = Tb[k] + (1.0 - lam) * S;
      }
    std::vector<int64_t> newc(nb);
    for (int r = 0; r < nb; ++r) {
      const int64_t c = ids[B[r]];
      int32_t h = hi;
      for (int q : b_side)
        if (M(B[r], q) != 0.0) h = std::min(h, chome[ids[q]]);
      cvert.push_back(cvert[c]);
      chome.push_back(h);
      cshare.push_back((1.0 - lam) * cshare[c]);
      cshare[c] *= lam;
      newc[r] = (int64_t)cvert.size() - 1;
      lines.push_back({c, newc[r]});
    }
    // alpha: I_a then B; beta: I_b then the new copies of B
    auto make = [&](const std::vector<int>& I, const std::vector<double>& Sx, std::vector<int64_t>& out_ids) {
      const int ni = (int)I.size();
      Dense D;
      D.n = ni + nb;
      D.a.assign((size_t)D.n * D.n, 0.0);
      for (int r = 0; r < ni; ++r) {
        for (int c = 0; c < ni; ++c) D(r, c) = M(I[r], I[c]);
        for (int c = 0; c < nb; ++c) D(r, ni + c) = D(ni + c, r) = M(I[r], B[c]);
      }
      for (int r = 0; r < nb; ++r)
        for (int c = 0; c < nb; ++c) D(ni + r, ni + c) = Sx[(size_t)r * nb + c];
      for (int r = 0; r < ni; ++r) out_ids.push_back(ids[I[r]]);
      return D;
    };
    std::vector<int64_t> ida, idb;
    Dense Ma = make(Ia, Sa, ida);
    for (int r = 0; r < nb; ++r) ida.push_back(ids[B[r]]);
    Dense Mb = make(Ib, Sb, idb);
    for (int r = 0; r < nb; ++r) idb.push_back(newc[r]);
    M = Dense();
    rec(std::move(ida), std::move(Ma), lo, mid);
    rec(std::move(idb), std::move(Mb), mid, hi);
  }
};

}  // namespace

constexpr int64_t kConformalMaxN = 8192;

void build_conformal(const vtm_partition_spec* sp, vtm_partition* p) {
  const int32_t N = sp->npieces;
  const int64_t n = p->n;
  if (N < 1 || !sp->home) fail(VTM_ERR_INVALID, "conformal: npieces >= 1 and home are required");
  if (!(sp->lambda > 0.0 && sp->lambda < 1.0)) fail(VTM_ERR_INVALID, "conformal: lambda must lie in (0, 1)");
  if (n > kConformalMaxN) fail(VTM_ERR_INVALID, "conformal: dense construction is limited to n <= 8192");
  std::vector<int64_t> cnt(N, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (sp->home[i] < 0 || sp->home[i] >= N) fail(VTM_ERR_INVALID, "conformal: home out of range");
    cnt[sp->home[i]]++;
  }
  for (int32_t q = 0; q < N; ++q)
    if (cnt[q] == 0) fail(VTM_ERR_INVALID, "conformal: every subgraph needs a home vertex");
  Builder b;
  b.lam = sp->lambda;
  b.cvert.resize(n);
  std::iota(b.cvert.begin(), b.cvert.end(), 0);
  b.chome.assign(sp->home, sp->home + n);
  b.cshare.assign(n, 1.0);
  b.piece_ids.resize(N);
  b.piece_mat.resize(N);
  Dense M0;
  M0.n = (int)n;
  M0.a.assign((size_t)n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = p->a_rowptr[i]; k < p->a_rowptr[i + 1]; ++k) M0((int)i, p->a_col[k]) += p->a_val[k];
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), 0);
  b.rec(std::move(all), std::move(M0), 0, N);

  // subgraphs in ascending vertex order; global copy ids numbered piece by piece
  p->npieces = N;
  p->piece_ptr.assign(N + 1, 0);
  std::vector<int64_t> gid(b.cvert.size(), -1);
  p->copy_vertex.clear();
  p->copy_share.clear();
  p->l_rowptr.assign(1, 0);
  p->l_col.clear();
  p->l_val.clear();
  std::vector<int64_t> vcount(n, 0);
  for (int32_t q = 0; q < N; ++q) {
    const auto& ids = b.piece_ids[q];
    const Dense& D = b.piece_mat[q];
    std::vector<int> ord(ids.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return b.cvert[ids[x]] < b.cvert[ids[y]]; });
    for (size_t r = 0; r < ord.size(); ++r) {
      const int64_t c = ids[ord[r]];
      gid[c] = (int64_t)p->copy_vertex.size();
      p->copy_vertex.push_back(b.cvert[c]);
      p->copy_share.push_back(b.cshare[c]);
      vcount[b.cvert[c]]++;
      for (size_t s2 = 0; s2 < ord.size(); ++s2) {
        const double v = D(ord[r], ord[s2]);
        if (v != 0.0) {
          p->l_col.push_back((int32_t)s2);
          p->l_val.push_back(v);
        }
      }
      p->l_rowptr.push_back((int64_t)p->l_col.size());
    }
    p->piece_ptr[q + 1] = (int64_t)p->copy_vertex.size();
  }
  p->line_a.clear();
  p->line_b.clear();
  for (const auto& ln : b.lines) {
    p->line_a.push_back(gid[ln.first]);
    p->line_b.push_back(gid[ln.second]);
  }
  int64_t nb = 0;
  for (int64_t i = 0; i < n; ++i) nb += vcount[i] > 1;
  p->nboundary = nb;
}

}  // namespace vtm
