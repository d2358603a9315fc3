// Solver setup and drivers behind vtm_setup / vtm_iterate / vtm_solve (host side).
//
// Setup (Table 1 steps 1-2, eq. 5.8): plan the band layout of every subgraph, sort the line ends
// by subgraph and port, upload Ã_j, assemble K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T on the device and
// factor it once.  Iteration (Table 1 steps 3-5): one k_sweep launch per sweep, ping-ponging the
// two wave buffers (the N2N exchange is the twin-indexed read of the previous buffer).
// Solve: sweeps plus the FP64 residual every check_every sweeps; FP32 solvers restart the sweeps
// on the FP64 residual (defect correction) once the inner residual has dropped enough or stalls.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <type_traits>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "kernels.h"

namespace vtm {

#define VTM_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) fail(VTM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  void alloc(size_t b) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = b;
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? VTM_ERR_OOM : VTM_ERR_CUDA,
           std::string("cudaMalloc(") + std::to_string(b) + "): " + cudaGetErrorString(e));
    }
  }
  void swap(DevBuf& o) {
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
  }
  template <class U>
  U* as() const {
    return static_cast<U*>(p);
  }
};

template <class U>
static void upload(DevBuf& d, const std::vector<U>& h, cudaStream_t st) {
  d.alloc(h.size() * sizeof(U));
  if (!h.empty()) VTM_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice, st));
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace vtm

using namespace vtm;

struct vtm_solver {
  int precision = VTM_FP64;
  int R = 1;
  int check_every = 10;
  double inner_reduction = 1e-4;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0, C = 0, E = 0;
  int32_t npieces = 0, nports = 0;
  size_t elem = 8;

  DevBuf pieces, factor, factor_u, bt, xc, w[2], port_local, port_end_ptr, twin, invz_t, status, port_rec;
  DevBuf a_rowptr, a_col, a_val, vc_ptr, vc_copy, copy_vertex, share;
  DevBuf vb, vx, vxt, vr, vrt, norms, nparts;  // nparts: per-block partial sums of the residual norms
  double* h_norms = nullptr;  // pinned: [R] residual^2, [R] b^2 ... plus status
  int cur = 0;                // wave buffer holding the last outgoing waves
  bool have_copies = false;
  int64_t launches = 0;       // kernels launched since creation (for accounting)

  std::vector<int32_t> api_to_int;  // end 2t+side -> internal (sorted) end
  int stages = 2;
  size_t sweep_smem = 0;
  int slot_elems = 0, ys_elems = 0, win_elems = 0;
  long wait_limit = 1L << 22;
  int withhold = -1;
  std::vector<int> stage_cands;
  // kept for re-assembly with new impedances (eq. 5.8 depends on Z)
  DevBuf d_copy_piece, d_lrowptr, d_lcol, d_lval, d_port_of_copy, d_invz64;
  std::vector<double> Z;             // per line, API order
  std::vector<int32_t> end_api;      // internal end -> API end (2t + side)
  std::vector<int32_t> end_port;     // internal end -> port
  int max_w = 0, max_pad = 0, max_ports = 0;
  bool wide = false;                 // R >= 16: windowed multi-RHS sweep kernel
  // FP32, every half-bandwidth <= 384: the tensor-core form of that sweep (sweep_wide_tc.cu)
  bool wt_ok = false, wide_tc = false;
  int64_t wt_bytes = 0;
  int wt_max_groups = 0;
  DevBuf wt;
  bool pipe = false;                 // R <= 2: pipelined sweep kernel chosen by the autotuner
  struct Cand {
    int stages;
    bool pipe;
  };
  std::vector<Cand> cands;
  int cap = 0;                       // its window rows
  std::vector<PieceDesc> pd_host;    // all subgraphs
  DevBuf pieces_lo;                  // subgraphs of the main launch (all, or the unflagged ones)
  int np_lo = 0;
  // FP32 solvers: subgraphs flagged by the FP32 factorisation, refactored and swept in FP64
  DevBuf hi_pieces, hi_factor, hi_factor_u;
  int np_hi = 0;
  int hi_stages = 2, hi_slot = 0, hi_ys = 0, hi_win = 0, hi_cap = 0;
  std::vector<int32_t> piece_bits;   // 32 or 64 per subgraph
  size_t hi_smem = 0;
  DevBuf hi_yspill;                  // R >= 16: FP64 forward results of the flagged subgraphs
  int64_t hi_rows = 0;               // sum of the flagged subgraphs' n_pad
  // port-response form (port.cu): S_j per subgraph, u_base per port, zero / scratch wave buffers
  bool port_form = false;
  bool port_tc = false;              // R >= 16, FP32: tensor-core port sweep (port_tc.cu)
  DevBuf S, ubase, wzero, wscr;
  bool ubase_ok = false;
  size_t port_smem = 0;
  bool port_det = false;             // SIMT port sweep: fixed-order (bitwise reproducible) reduction
  DevBuf S16, sig16, tc_scratch;     // tensor-core form: fp16 hi / lo blocks, sigma_j, s^T slots
  DevBuf gscale;                     // tensor-core form: sqrt(S_pp) per port (diagonal balance)
  int tc_grid = 0, tc_n4max = 0, tc_tmem_cols = 0;
  int64_t tc_bytes_hi = 0, tc_bytes_all = 0;  // bytes a sweep streams without / with the lo half
  DevBuf Sh, hscale;                 // FP16 copy of S_j and the scale of each of its tiles
  bool port_half = false;            // the port sweep reads the FP16 copy (tensor cores: hi half only)
  bool port_half_auto = false;       // ... and returns to FP32 when a correction step stalls
  // coupled lines (§7.2): per-port coupling lists, read by the sweep kernels' port loops
  bool coupled = false;
  DevBuf cp_ptr, cp_oth, cp_y;
  std::vector<double> ydiag;         // per line: sum of its coupling conductances (diagonal of Y)
  // the last vtm_solve's residual checks: sweeps so far, max relative residual, max inner residual
  std::vector<int32_t> hist_sweeps;
  std::vector<double> hist_rel, hist_inner;
  vtm_solver_info info{};

  // captured CUDA graphs of k back-to-back sweeps, keyed by (k, starting wave buffer)
  struct Graph {
    int k, cur;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  bool use_graphs = true;

  ~vtm_solver() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    if (h_norms) cudaFreeHost(h_norms);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace vtm {

// NVTX range for the phases of setup and solve (visible to ncu --nvtx and other NVTX tools).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

static void check_status(vtm_solver* s) {
  int st = 0;
  VTM_CUDA(cudaMemcpyAsync(&st, s->status.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
  if (st == kStatusTimeout) fail(VTM_ERR_TIMEOUT, "a bounded device wait ran out in the sweep kernel");
  if (st == kStatusNotSpd) fail(VTM_ERR_NOT_SPD, "a local matrix K_j had a non-positive Cholesky pivot");
  if (st != 0) fail(VTM_ERR_INVALID, "device status " + std::to_string(st));
}

// Restart threshold of a defect-correction phase swept on FP16 port responses: 4 units of 2^-11.
constexpr double kHalfReduction = 4.0 / 2048.0;

template <typename T>
static void autotune_sweep(vtm_solver* s);
template <typename T>
static void choose_form(vtm_solver* s, const vtm_setup_opts* o, int64_t s_tiles, int64_t band_elems);
void reset_waves(vtm_solver* s);

static size_t sweep_smem_for(const vtm_solver* s, size_t elem, int stages, bool pipe = false) {
  if (s->wide) return sweep_wide_smem_bytes(elem, s->R, stages, s->slot_elems, s->cap);
  if (pipe) return sweep_pipe_smem_bytes(elem, s->R, stages, s->slot_elems, s->ys_elems, s->win_elems);
  return sweep_smem_bytes(elem, s->R, stages, s->slot_elems, s->ys_elems, s->win_elems);
}
void line_features(const vtm_partition* p, float* out);
void mlp_forward(const vtm_mlp* m, const float* X, float* y, int64_t n, cudaStream_t st);

// Assemble K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T for the solver's current line impedances and factor
// every K_j on the device (eq. 5.8, once per choice of Z).
// Assemble K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T for the solver's line impedances and factor every
// K_j on the device once (eq. 5.8).  FP32 solvers flag the subgraphs whose FP32 factorisation broke
// down or lost most of its digits, and refactor those in FP64 (their own band, swept by an FP64
// instance of the sweep kernel).
template <typename T>
static void factor_typed(vtm_solver* s) {
  cudaStream_t st = s->stream;
  const int np = s->npieces;
  std::vector<double> invz(s->E);
  for (int64_t k = 0; k < s->E; ++k) {
    const int32_t t = s->end_api[k] >> 1;
    invz[k] = 1.0 / s->Z[t] + (s->ydiag.empty() ? 0.0 : s->ydiag[t]);  // diagonal of Y (§7.2)
  }
  upload(s->d_invz64, invz, st);
  {
    std::vector<T> iz(invz.begin(), invz.end());
    upload(s->invz_t, iz, st);
  }
  VTM_CUDA(cudaMemsetAsync(s->factor.p, 0, s->factor.bytes, st));
  VTM_CUDA(launch_build_band<T>(s->C, s->d_copy_piece.as<int32_t>(), s->pieces.as<PieceDesc>(),
                                s->d_lrowptr.as<int64_t>(), s->d_lcol.as<int32_t>(), s->d_lval.as<double>(),
                                s->d_port_of_copy.as<int32_t>(), s->port_end_ptr.as<int32_t>(),
                                s->d_invz64.as<double>(), np, s->max_pad, s->factor.as<T>(),
                                s->status.as<int>(), st));
  const bool flagging = sizeof(T) == 4;
  DevBuf flags, diag0;
  if (flagging) {
    flags.alloc((size_t)np * sizeof(int));
    VTM_CUDA(cudaMemsetAsync(flags.p, 0, flags.bytes, st));
    diag0.alloc((size_t)(s->pd_host.back().row_off + s->pd_host.back().n_pad) * sizeof(T));
  }
  cudaEvent_t e0, e1;
  VTM_CUDA(cudaEventCreate(&e0));
  VTM_CUDA(cudaEventCreate(&e1));
  VTM_CUDA(cudaEventRecord(e0, st));
  cudaError_t fe;
  bool tc_factor = false;
  if constexpr (sizeof(T) == 4) {
    // wide bands: the trailing update is a sizeable dense product, run on the tensor cores
    tc_factor = s->max_w >= 64 && s->max_w <= 384 && factor_tc_smem_bytes(s->max_w) <= 227 * 1024;
    if (tc_factor)
      fe = launch_factor_tc(s->pieces.as<PieceDesc>(), np, s->max_w, s->factor.as<float>(), s->status.as<int>(),
                            flags.as<int>(), diag0.as<float>(), s->wait_limit, st);
  }
  if (!tc_factor)
    fe = launch_factor<T>(s->pieces.as<PieceDesc>(), np, s->max_w, s->factor.as<T>(), s->status.as<int>(),
                          flagging ? flags.as<int>() : nullptr, flagging ? diag0.as<T>() : nullptr, st);
  s->info.factor_tc = tc_factor ? 1 : 0;
  VTM_CUDA(cudaEventRecord(e1, st));
  VTM_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (fe == cudaErrorInvalidValue) fail(VTM_ERR_INVALID, "bandwidth too large for the factorisation kernel");
  VTM_CUDA(fe);
  s->info.factor_ms += ms;
  check_status(s);
  if (!s->wide) {
    VTM_CUDA(launch_transpose_band<T>(s->pieces.as<PieceDesc>(), np, s->factor.as<T>(), s->factor_u.as<T>(), st));
    VTM_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int> fl(np, 0);
  if (flagging) VTM_CUDA(cudaMemcpy(fl.data(), flags.p, np * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<PieceDesc> lo, hi;
  std::vector<int32_t> hi_of_piece(np, -1);
  int64_t hoff = 0, hrows = 0;
  int max_w_hi = 0;
  for (int j = 0; j < np; ++j) {
    if (!fl[j]) {
      lo.push_back(s->pd_host[j]);
      continue;
    }
    PieceDesc d = s->pd_host[j];
    int Wp = std::max(d.w + 1, kNB);
    while (Wp % 16 != 4) ++Wp;
    d.Wp = Wp;
    d.factor_off = hoff;
    d.row_off = hrows;  // rows of this piece in the FP64 spill buffer of the multi-RHS sweep
    hrows += d.n_pad;
    hoff += (int64_t)d.n_pad * Wp;
    hi_of_piece[j] = (int32_t)hi.size();
    max_w_hi = std::max(max_w_hi, d.w);
    hi.push_back(d);
  }
  s->np_lo = (int)lo.size();
  s->np_hi = (int)hi.size();
  s->piece_bits.assign(np, sizeof(T) == 8 ? 64 : 32);
  for (int j = 0; j < np; ++j)
    if (fl[j]) s->piece_bits[j] = 64;
  s->info.flagged_pieces = s->np_hi;
  if (!lo.empty()) upload(s->pieces_lo, lo, st);
  if (hi.empty()) return;
  // FP64 band of the flagged subgraphs
  std::vector<int32_t> cp(s->C, -1);
  for (int j = 0; j < np; ++j)
    if (hi_of_piece[j] >= 0)
      for (int64_t c = s->pd_host[j].copy_off; c < s->pd_host[j].copy_off + s->pd_host[j].n; ++c) cp[c] = hi_of_piece[j];
  DevBuf dcp;
  upload(dcp, cp, st);
  upload(s->hi_pieces, hi, st);
  s->hi_factor.alloc((size_t)hoff * sizeof(double));
  s->hi_rows = hrows;
  if (s->wide) s->hi_yspill.alloc((size_t)hrows * s->R * sizeof(double));
  VTM_CUDA(cudaMemsetAsync(s->hi_factor.p, 0, s->hi_factor.bytes, st));
  int max_pad_hi = 0;
  for (const auto& d : hi) max_pad_hi = std::max(max_pad_hi, d.n_pad);
  VTM_CUDA(launch_build_band<double>(s->C, dcp.as<int32_t>(), s->hi_pieces.as<PieceDesc>(), s->d_lrowptr.as<int64_t>(),
                                     s->d_lcol.as<int32_t>(), s->d_lval.as<double>(), s->d_port_of_copy.as<int32_t>(),
                                     s->port_end_ptr.as<int32_t>(), s->d_invz64.as<double>(), s->np_hi, max_pad_hi,
                                     s->hi_factor.as<double>(), s->status.as<int>(), st));
  VTM_CUDA(launch_factor<double>(s->hi_pieces.as<PieceDesc>(), s->np_hi, max_w_hi, s->hi_factor.as<double>(),
                                 s->status.as<int>(), nullptr, nullptr, st));
  VTM_CUDA(cudaStreamSynchronize(st));
  check_status(s);
  if (!s->wide) {
    s->hi_factor_u.alloc((size_t)hoff * sizeof(double));
    VTM_CUDA(launch_transpose_band<double>(s->hi_pieces.as<PieceDesc>(), s->np_hi, s->hi_factor.as<double>(),
                                           s->hi_factor_u.as<double>(), st));
    VTM_CUDA(cudaStreamSynchronize(st));
  }
}

template <typename T>
static void input_impedances_typed(vtm_solver* s, std::vector<double>& r_api);

// Shared-memory plan of the FP64 launch over the flagged subgraphs (FP64 factor, FP32 vectors).
static void plan_hi(vtm_solver* s) {
  if (s->np_hi == 0) return;
  std::vector<PieceDesc> hi(s->np_hi);
  VTM_CUDA(cudaMemcpy(hi.data(), s->hi_pieces.p, hi.size() * sizeof(PieceDesc), cudaMemcpyDeviceToHost));
  int mWp = 0, mpad = 0, mends = 0;
  for (const auto& d : hi) {
    mWp = std::max(mWp, d.Wp);
    mpad = std::max(mpad, d.n_pad);
    mends = std::max(mends, d.nends);
  }
  const int R = s->R;
  s->hi_slot = kNB * mWp;
  s->hi_ys = (2 * (mWp - 1) + mpad) * R;
  s->hi_win = std::max(1, mends) * R;
  s->hi_cap = 64;
  while (s->hi_cap < mWp - 1 + kNB) s->hi_cap *= 2;
  if (s->wide && s->hi_cap > kWideWindow) fail(VTM_ERR_INVALID, "flagged subgraph too wide for the multi-RHS window");
  const size_t kSmemMax = 227 * 1024;
  s->hi_stages = 0;
  for (int st2 : {8, 6, 4, 3, 2}) {
    if (s->hi_stages) break;
    const size_t b = s->wide ? sweep_wide_smem_bytes(sizeof(double), R, st2, s->hi_slot, s->hi_cap)
                             : sweep_smem_bytes(sizeof(double), R, st2, s->hi_slot, s->hi_ys, s->hi_win);
    if (b <= kSmemMax) {
      s->hi_stages = st2;
      s->hi_smem = b;
    }
  }
  if (!s->hi_stages) fail(VTM_ERR_INVALID, "a subgraph flagged for FP64 is too large for the FP64 sweep");
  if (s->wide) VTM_CUDA((sweep_wide_configure<double, float>(R, s->hi_smem)));
  else VTM_CUDA((sweep_configure<double, float>(R, s->hi_smem)));
}

// Coupled lines (§7.2): check every pair; the diagonal of Y (1/Z_t + the line's conductances) goes
// into the per-end 1/Z array (ydiag), the off-diagonal -y into the local matrix values of both
// subgraphs, so that K_j = Ã_j + P_j Y_j P_j^T comes out of the usual assembly; list per port the
// incoming wave and the off-diagonal admittance of each coupling (CoupleRef).
template <typename T>
static void couple_setup(const vtm_partition* p, const vtm_setup_opts* o, vtm_solver* s,
                         const std::vector<int32_t>& copy_piece, const std::vector<int32_t>& port_end_ptr,
                         const std::vector<int32_t>& twin, std::vector<double>& lval) {
  if (!o->couplings || !o->coupling_y) fail(VTM_ERR_INVALID, "couplings or coupling_y is NULL");
  const int64_t nl = (int64_t)p->line_a.size();
  std::vector<int32_t> eport(2 * nl, 0);
  for (size_t q = 0; q + 1 < port_end_ptr.size(); ++q)
    for (int32_t e = port_end_ptr[q]; e < port_end_ptr[q + 1]; ++e) eport[e] = (int32_t)q;
  auto find = [&](int64_t c, int64_t lc) -> int64_t {
    for (int64_t k = p->l_rowptr[c]; k < p->l_rowptr[c + 1]; ++k)
      if (p->l_col[k] == lc) return k;
    return -1;
  };
  struct Ent {
    int32_t port, oth;
    double y;
  };
  s->ydiag.assign(nl, 0.0);
  std::vector<Ent> ent;
  int64_t used = 0;
  for (int64_t k = 0; k < o->ncouplings; ++k) {
    const int64_t t = o->couplings[2 * k], u = o->couplings[2 * k + 1];
    const double y = o->coupling_y[k];
    if (t < 0 || u < 0 || t >= nl || u >= nl) fail(VTM_ERR_INVALID, "coupled line id out of range");
    if (t == u) fail(VTM_ERR_INVALID, "a line cannot be coupled with itself");
    if (!(y >= 0) || !std::isfinite(y)) fail(VTM_ERR_INVALID, "coupling conductances must be >= 0 and finite");
    const int32_t ja = copy_piece[p->line_a[t]], jb = copy_piece[p->line_b[t]];
    const int32_t ka = copy_piece[p->line_a[u]], kb = copy_piece[p->line_b[u]];
    if (!((ja == ka && jb == kb) || (ja == kb && jb == ka)))
      fail(VTM_ERR_INVALID, "coupled lines must join the same two subgraphs");
    if (y == 0) continue;
    ++used;
    s->ydiag[t] += y;
    s->ydiag[u] += y;
    for (int side = 0; side < 2; ++side) {
      const int32_t j = side ? jb : ja;
      const int64_t ct = side ? p->line_b[t] : p->line_a[t];
      const int us = copy_piece[p->line_a[u]] == j ? 0 : 1;
      const int64_t cu = us ? p->line_b[u] : p->line_a[u];
      if (ct == cu) fail(VTM_ERR_INVALID, "coupled lines end at the same copy");
      const int64_t lt = ct - p->piece_ptr[j], lu = cu - p->piece_ptr[j];
      const int64_t k1 = find(ct, lu), k2 = find(cu, lt);
      if (k1 < 0 || k2 < 0) fail(VTM_ERR_INVALID, "coupled lines must join neighbouring copies in both subgraphs");
      lval[k1] -= y;
      lval[k2] -= y;
      const int32_t it = s->api_to_int[2 * t + side], iu = s->api_to_int[2 * u + us];
      ent.push_back({eport[it], twin[iu], -y});
      ent.push_back({eport[iu], twin[it], -y});
    }
  }
  // CSR by port, entries of a port in the order they were made (a counting sort: millions of pairs)
  const int nports = (int)port_end_ptr.size() - 1;
  std::vector<int32_t> ptr(nports + 1, 0), oth(ent.size());
  std::vector<T> yv(ent.size());
  for (const Ent& x : ent) ptr[x.port + 1]++;
  for (int q = 0; q < nports; ++q) ptr[q + 1] += ptr[q];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (const Ent& x : ent) {
      const int32_t at = fill[x.port]++;
      oth[at] = x.oth;
      yv[at] = (T)x.y;
    }
  }
  s->info.ncouplings = used;
  if (used == 0) {
    s->ydiag.clear();
    return;
  }
  s->coupled = true;
  upload(s->cp_ptr, ptr, s->stream);
  upload(s->cp_oth, oth, s->stream);
  upload(s->cp_y, yv, s->stream);
}

// The tensor-core factor of the subgraphs of the main launch (FP32 band factor -> balanced fp16
// panels), when every half-bandwidth allows it and it fits in device memory with room to spare.
static bool build_wide_tc(vtm_solver* s) {
  if (!s->wt_ok || s->np_lo == 0) return false;
  size_t free_b = 0, total_b = 0;
  VTM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  if ((double)s->wt_bytes > 0.6 * (double)free_b) return false;
  s->wt.alloc((size_t)s->wt_bytes);
  VTM_CUDA(cudaMemsetAsync(s->wt.p, 0, (size_t)wide_tc_zero_bytes(), s->stream));
  VTM_CUDA(wide_tc_configure(s->R));
  VTM_CUDA(launch_wide_tc_factor(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->wt_max_groups, s->factor.as<float>(),
                                 s->wt.as<unsigned char>(), s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
  s->info.band_tc = 1;
  s->info.band_tc_bytes = s->wt_bytes;
  return true;
}

template <typename T>
static void setup_typed(const vtm_partition* p, const vtm_setup_opts* o, vtm_solver* s) {
  cudaStream_t st = s->stream;
  const int32_t np = p->npieces;
  const int64_t C = p->piece_ptr[np];
  const int64_t nl = (int64_t)p->line_a.size();
  s->n = p->n;
  s->C = C;
  s->E = 2 * nl;
  s->npieces = np;
  s->elem = sizeof(T);
  s->wide = s->R >= 16;

  // ---- impedances per line
  std::vector<double> Z(nl);
  for (int64_t t = 0; t < nl; ++t) {
    double z = (o->z_mode == VTM_Z_EXPLICIT) ? o->z_lines[t] : o->z_uniform;  // MATCHED starts from z_uniform
    if (o->z_mode == VTM_Z_LEARNED) z = 1.0;
    if (!(z > 0) || !std::isfinite(z)) fail(VTM_ERR_INVALID, "line impedances must be positive and finite");
    Z[t] = z;
  }
  if (o->z_mode == VTM_Z_LEARNED && nl > 0) {
    // the model proposes log Z for each end; both ends agree on the geometric mean (Table 1 step 1)
    std::vector<float> feats((size_t)2 * nl * VTM_MLP_IN), y(2 * nl);
    line_features(p, feats.data());
    DevBuf dX, dy;
    upload(dX, feats, st);
    dy.alloc(y.size() * sizeof(float));
    mlp_forward(o->model, dX.as<float>(), dy.as<float>(), 2 * nl, st);
    VTM_CUDA(cudaMemcpyAsync(y.data(), dy.p, y.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    VTM_CUDA(cudaStreamSynchronize(st));
    for (int64_t t = 0; t < nl; ++t) {
      double lz = 0.5 * ((double)y[2 * t] + (double)y[2 * t + 1]);
      if (!std::isfinite(lz)) fail(VTM_ERR_INVALID, "learned impedance is not finite");
      lz = std::min(30.0, std::max(-30.0, lz));
      Z[t] = std::exp(lz);
    }
  }

  // ---- ends sorted by (copy, line, side); copies are grouped by subgraph in local order
  std::vector<int64_t> end_copy(2 * nl);
  for (int64_t t = 0; t < nl; ++t) {
    end_copy[2 * t] = p->line_a[t];
    end_copy[2 * t + 1] = p->line_b[t];
  }
  std::vector<int32_t> order(2 * nl);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return end_copy[a] < end_copy[b]; });
  s->api_to_int.assign(2 * nl, 0);
  for (int64_t k = 0; k < 2 * nl; ++k) s->api_to_int[order[k]] = (int32_t)k;
  std::vector<int32_t> twin(2 * nl);
  std::vector<double> invz(2 * nl);
  for (int64_t k = 0; k < 2 * nl; ++k) {
    const int32_t api = order[k];
    twin[k] = s->api_to_int[api ^ 1];
    invz[k] = 1.0 / Z[api >> 1];
  }
  // ports: distinct copies among the sorted ends
  std::vector<int32_t> port_local, port_end_ptr;
  std::vector<int32_t> port_of_copy(C, -1);
  std::vector<int32_t> copy_piece(C);
  for (int32_t j = 0; j < np; ++j)
    for (int64_t c = p->piece_ptr[j]; c < p->piece_ptr[j + 1]; ++c) copy_piece[c] = j;
  std::vector<PieceDesc> pd(np);
  for (int32_t j = 0; j < np; ++j) {
    pd[j].nports = 0;
    pd[j].nends = 0;
    pd[j].port_off = 0;
    pd[j].end_off = 0;
  }
  {
    int64_t k = 0;
    int32_t lastpiece = -1;
    while (k < 2 * nl) {
      const int64_t c = end_copy[order[k]];
      const int32_t j = copy_piece[c];
      if (j != lastpiece) {
        pd[j].port_off = (int32_t)port_local.size();
        pd[j].end_off = (int32_t)k;
        lastpiece = j;
      }
      port_of_copy[c] = (int32_t)port_local.size();
      port_local.push_back((int32_t)(c - p->piece_ptr[j]));
      port_end_ptr.push_back((int32_t)k);
      int64_t k2 = k;
      while (k2 < 2 * nl && end_copy[order[k2]] == c) ++k2;
      pd[j].nports++;
      pd[j].nends += (int32_t)(k2 - k);
      k = k2;
    }
    port_end_ptr.push_back((int32_t)(2 * nl));
  }
  s->nports = (int32_t)port_local.size();
  // pieces without ports still need a valid port_off/end_off
  for (int32_t j = 0; j < np; ++j)
    if (pd[j].nports == 0) {
      pd[j].port_off = 0;
      pd[j].end_off = 0;
    }

  // ---- band layout
  const int wmod = (sizeof(T) == 4) ? 32 : 16, wrem = (sizeof(T) == 4) ? 8 : 4;
  int64_t foff = 0, band_entries = 0, row_total = 0, soff = 0;
  int max_w = 0, max_Wp = 0, max_pad = 0, max_ends = 0;
  for (int32_t j = 0; j < np; ++j) {
    const int64_t n_j = p->piece_ptr[j + 1] - p->piece_ptr[j];
    if (n_j > (1 << 30)) fail(VTM_ERR_INVALID, "subgraph too large");
    int w = 0;
    for (int64_t c = p->piece_ptr[j]; c < p->piece_ptr[j + 1]; ++c) {
      const int64_t l = c - p->piece_ptr[j];
      for (int64_t k = p->l_rowptr[c]; k < p->l_rowptr[c + 1]; ++k) w = std::max<int64_t>(w, std::llabs(l - p->l_col[k]));
    }
    int Wp = std::max(w + 1, kNB);
    while (Wp % wmod != wrem) ++Wp;
    const int n_pad = (int)((n_j + kNB - 1) / kNB) * kNB;
    pd[j].factor_off = foff;
    pd[j].row_off = row_total;
    row_total += (int64_t)((n_j + kNB - 1) / kNB) * kNB;
    pd[j].copy_off = p->piece_ptr[j];
    pd[j].n = (int32_t)n_j;
    pd[j].n_pad = n_pad;
    pd[j].Wp = Wp;
    pd[j].w = w;
    foff += (int64_t)n_pad * Wp;
    pd[j].s_off = soff;
    soff += port_tiles(pd[j].nports);
    band_entries += n_j * (w + 1) - (int64_t)w * (w + 1) / 2;
    max_w = std::max(max_w, w);
    max_Wp = std::max(max_Wp, Wp);
    max_pad = std::max(max_pad, n_pad);
    max_ends = std::max(max_ends, pd[j].nends);
  }
  if (sizeof(T) == 4 && o->sweep_variant != 3) {
    s->wt_ok = true;
    s->wt_bytes = wide_tc_zero_bytes();
    for (int32_t j = 0; j < np; ++j) {
      if (!wide_tc_fits(pd[j].w)) s->wt_ok = false;
      pd[j].wt_off = s->wt_bytes;
      s->wt_bytes += wide_tc_bytes(pd[j].n, pd[j].w);
      s->wt_max_groups = std::max(s->wt_max_groups, wide_tc_groups(pd[j].n));
    }
  }

  // ---- sweep shared-memory plan: every staging depth that fits is a tuning candidate
  const int R = s->R;
  s->slot_elems = kNB * max_Wp;
  s->ys_elems = (2 * (max_Wp - 1) + max_pad) * R;
  s->win_elems = std::max(1, max_ends) * R;
  const size_t kSmemMax = 227 * 1024;
  std::vector<int> stage_cands;
  size_t smem_cap = 0;
  if (s->wide && max_Wp - 1 + kNB > kWideWindow)
    fail(VTM_ERR_INVALID, "bandwidth too large for the multi-RHS sweep window");
  s->cap = 64;
  while (s->cap < max_Wp - 1 + kNB) s->cap *= 2;
  // deeper rings for thin bands: a slab of a 2D subgraph is a few KB, and hiding DRAM latency takes
  // several of them in flight (the mbarrier area holds up to kMaxStages)
  size_t pipe_cap = 0;
  for (int st2 : {2, 3, 4, 6, 8, 12, kMaxStages}) {
    const size_t b = sweep_smem_for(s, sizeof(T), st2, false);
    if (b <= kSmemMax) {
      stage_cands.push_back(st2);
      if (o->sweep_variant != 2) s->cands.push_back({st2, false});
      smem_cap = std::max(smem_cap, b);
    }
    // the pipelined schedule measured slower than the single-block one on every workload tried, so
    // the autotuner only considers it when it is asked for explicitly
    if (!s->wide && R <= 2 && st2 >= 3 && o->sweep_variant == 2) {
      const size_t bp = sweep_smem_for(s, sizeof(T), st2, true);
      if (bp <= kSmemMax) {
        s->cands.push_back({st2, true});
        pipe_cap = std::max(pipe_cap, bp);
      }
    }
  }
  if (stage_cands.empty())
    fail(VTM_ERR_INVALID, "a subgraph is too large for the shared-memory sweep (n_j, bandwidth or nrhs too big)");
  if (s->cands.empty())
    fail(VTM_ERR_INVALID, "the requested sweep variant is not available for this nrhs and subgraph size");
  s->stage_cands = stage_cands;
  s->stages = stage_cands.back();
  s->sweep_smem = sweep_smem_for(s, sizeof(T), s->stages);
  if (s->wide) VTM_CUDA((sweep_wide_configure<T, T>(R, smem_cap)));
  else VTM_CUDA((sweep_configure<T, T>(R, smem_cap)));
  if (pipe_cap > 0) VTM_CUDA((sweep_pipe_configure<T, T>(R, pipe_cap)));

  // ---- vertex -> copies (for assembly)
  std::vector<int64_t> vc_ptr(p->n + 1, 0), vc_copy(C);
  for (int64_t c = 0; c < C; ++c) vc_ptr[p->copy_vertex[c] + 1]++;
  for (int64_t i = 0; i < p->n; ++i) vc_ptr[i + 1] += vc_ptr[i];
  {
    std::vector<int64_t> fill(vc_ptr.begin(), vc_ptr.end() - 1);
    for (int64_t c = 0; c < C; ++c) vc_copy[fill[p->copy_vertex[c]]++] = c;
  }

  // ---- device buffers
  upload(s->pieces, pd, st);
  s->pd_host = pd;
  upload(s->port_local, port_local, st);
  upload(s->port_end_ptr, port_end_ptr, st);
  upload(s->twin, twin, st);
  upload(s->a_rowptr, p->a_rowptr, st);
  upload(s->a_col, p->a_col, st);
  upload(s->a_val, p->a_val, st);
  upload(s->vc_ptr, vc_ptr, st);
  upload(s->vc_copy, vc_copy, st);
  upload(s->copy_vertex, p->copy_vertex, st);
  upload(s->share, p->copy_share, st);
  s->status.alloc(sizeof(int));
  VTM_CUDA(cudaMemsetAsync(s->status.p, 0, sizeof(int), st));

  // local matrices and factor
  upload(s->d_copy_piece, copy_piece, st);
  upload(s->d_lrowptr, p->l_rowptr, st);
  upload(s->d_lcol, p->l_col, st);
  if (o->ncouplings > 0) {
    std::vector<double> lval = p->l_val;
    couple_setup<T>(p, o, s, copy_piece, port_end_ptr, twin, lval);
    upload(s->d_lval, lval, st);
  } else {
    if (o->ncouplings < 0) fail(VTM_ERR_INVALID, "ncouplings must be >= 0");
    upload(s->d_lval, p->l_val, st);
  }
  upload(s->d_port_of_copy, port_of_copy, st);
  s->factor.alloc((size_t)foff * sizeof(T));
  if (!s->wide) s->factor_u.alloc((size_t)foff * sizeof(T));
  s->max_w = max_w;
  s->max_pad = max_pad;
  s->Z = Z;
  s->end_api = order;
  s->end_port.assign(2 * nl, 0);
  for (size_t q = 0; q + 1 < port_end_ptr.size(); ++q)
    for (int32_t e = port_end_ptr[q]; e < port_end_ptr[q + 1]; ++e) s->end_port[e] = (int32_t)q;
  for (int32_t j = 0; j < np; ++j) s->max_ports = std::max(s->max_ports, pd[j].nports);
  {
    Range r("vtm_setup/factor");
    factor_typed<T>(s);
  }
  plan_hi(s);
  if constexpr (sizeof(T) == 4) {
    if (s->wide && build_wide_tc(s)) s->wide_tc = true;
  }

  // vectors
  s->bt.alloc((size_t)C * R * sizeof(T));
  s->xc.alloc((size_t)C * R * sizeof(T));
  for (int b = 0; b < 2; ++b) {
    s->w[b].alloc((size_t)std::max<int64_t>(1, s->E) * R * sizeof(T));
    VTM_CUDA(cudaMemsetAsync(s->w[b].p, 0, s->w[b].bytes, st));
  }
  VTM_CUDA(cudaMemsetAsync(s->bt.p, 0, s->bt.bytes, st));
  VTM_CUDA(cudaMemsetAsync(s->xc.p, 0, s->xc.bytes, st));
  const size_t nv = (size_t)p->n * R * sizeof(double);
  s->vb.alloc(nv);
  s->vx.alloc(nv);
  s->vxt.alloc(nv);
  s->vr.alloc(nv);
  s->vrt.alloc(nv);
  s->norms.alloc(2 * kMaxRhs * sizeof(double));
  s->nparts.alloc((size_t)norm_parts(p->n) * R * sizeof(double));
  VTM_CUDA(cudaMallocHost(&s->h_norms, 2 * kMaxRhs * sizeof(double)));
  VTM_CUDA(cudaStreamSynchronize(st));

  {
    Range r("vtm_setup/autotune");
    autotune_sweep<T>(s);
  }
  {
    Range r("vtm_setup/form");
    choose_form<T>(s, o, soff, foff);
  }
  s->withhold = o->withhold_slab > 0 ? o->withhold_slab - 1 : -1;  // after tuning: only real sweeps

  s->info.npieces = np;
  s->info.ncopies = C;
  s->info.nends = s->E;
  s->info.nports = s->nports;
  s->info.nrhs = R;
  s->info.precision = s->precision;
  s->info.block_rows = kNB;
  s->info.factor_entries = foff;
  s->info.band_entries = band_entries;
  s->info.factor_bytes = foff * (int64_t)sizeof(T);
  s->info.max_halfband = max_w;
}

template <typename TV>
static CoupleRef<TV> couple_ref(vtm_solver* s) {
  CoupleRef<TV> c{};
  if (s->coupled) {
    c.ptr = s->cp_ptr.as<int32_t>();
    c.oth = s->cp_oth.as<int32_t>();
    c.y = s->cp_y.as<TV>();
  }
  return c;
}

template <typename TF, typename TV>
static SweepArgs<TF, TV> sweep_args(vtm_solver* s, int write_x, bool hi) {
  SweepArgs<TF, TV> a;
  a.pieces = hi ? s->hi_pieces.as<PieceDesc>() : s->pieces_lo.as<PieceDesc>();
  a.factor = hi ? s->hi_factor.as<TF>() : s->factor.as<TF>();
  a.factor_u = hi ? s->hi_factor_u.as<TF>() : s->factor_u.as<TF>();
  a.bt = s->bt.as<TV>();
  a.xc = s->xc.as<TV>();
  a.wprev = s->w[s->cur].as<TV>();
  a.wnext = s->w[s->cur ^ 1].as<TV>();
  a.port_local = s->port_local.as<int32_t>();
  a.port_end_ptr = s->port_end_ptr.as<int32_t>();
  a.twin = s->twin.as<int32_t>();
  a.invz = s->invz_t.as<TV>();
  a.status = s->status.as<int>();
  a.write_x = write_x;
  a.stages = hi ? s->hi_stages : s->stages;
  a.slot_elems = hi ? s->hi_slot : s->slot_elems;
  a.ys_elems = hi ? s->hi_ys : s->ys_elems;
  a.win_elems = hi ? s->hi_win : s->win_elems;
  a.wait_limit = s->wait_limit;
  a.withhold = s->withhold;
  a.cap = hi ? s->hi_cap : s->cap;
  a.yspill = (hi && s->wide) ? s->hi_yspill.as<TF>() : nullptr;
  a.cpl = couple_ref<TV>(s);
  a.wt = (!hi && s->wide_tc) ? s->wt.as<unsigned char>() : nullptr;
  return a;
}

template <typename TF, typename TV>
static void launch_one(vtm_solver* s, const SweepArgs<TF, TV>& a, int np, size_t smem, bool pipe) {
  if constexpr (std::is_same_v<TF, float> && std::is_same_v<TV, float>) {
    if (s->wide && a.wt) {
      VTM_CUDA(launch_sweep_wide_tc(a, s->R, np, s->stream));
      s->launches++;
      return;
    }
  }
  if (s->wide) VTM_CUDA((launch_sweep_wide<TF, TV>(a, s->R, np, smem, s->stream)));
  else if (pipe) VTM_CUDA((launch_sweep_pipe<TF, TV>(a, s->R, np, smem, s->stream)));
  else VTM_CUDA((launch_sweep<TF, TV>(a, s->R, np, smem, s->stream)));
  s->launches++;
}

template <typename T>
static void sweeps_typed(vtm_solver* s, int k) {
  for (int i = 0; i < k; ++i) {
    const int wx = i == k - 1;
    if (s->np_lo > 0) launch_one<T, T>(s, sweep_args<T, T>(s, wx, false), s->np_lo, s->sweep_smem, s->pipe);
    if constexpr (sizeof(T) == 4) {
      if (s->np_hi > 0)
        launch_one<double, float>(s, sweep_args<double, float>(s, wx, true), s->np_hi, s->hi_smem, false);
    }
    s->cur ^= 1;
  }
  if (k > 0) s->have_copies = true;
}

// Setup-time autotuner: time each staging depth that fits (fewer stages leave room for more
// resident CTAs per SM) on the solver's own subgraphs and keep the fastest.
template <typename T>
static void autotune_sweep(vtm_solver* s) {
  cudaEvent_t e0, e1;
  VTM_CUDA(cudaEventCreate(&e0));
  VTM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_st = s->stage_cands.back();
  bool best_pipe = false;
  // the tensor-core multi-RHS sweep has no staging depth to choose: time it once
  const std::vector<vtm_solver::Cand> cands = s->wide_tc ? std::vector<vtm_solver::Cand>{{best_st, false}} : s->cands;
  for (const auto& c : cands) {
    s->stages = c.stages;
    s->pipe = c.pipe;
    s->sweep_smem = sweep_smem_for(s, sizeof(T), c.stages, c.pipe);
    sweeps_typed<T>(s, 1);
    VTM_CUDA(cudaEventRecord(e0, s->stream));
    sweeps_typed<T>(s, 3);  // direct launches: the configuration is still being chosen
    VTM_CUDA(cudaEventRecord(e1, s->stream));
    VTM_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    VTM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 3;
    if (ms < best) {
      best = ms;
      best_st = c.stages;
      best_pipe = c.pipe;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->stages = best_st;
  s->pipe = best_pipe;
  s->sweep_smem = sweep_smem_for(s, sizeof(T), best_st, best_pipe);
  s->info.sweep_variant = best_pipe ? 1 : 0;
  int occ = 1;
  if (!s->wide && !s->pipe) VTM_CUDA((sweep_occupancy<T, T>(s->R, s->sweep_smem, &occ)));
  if (s->pipe) VTM_CUDA((sweep_pipe_occupancy<T, T>(s->R, s->sweep_smem, &occ)));
  s->info.sweep_stages = best_st;
  s->info.sweep_ctas_per_sm = occ;
  s->info.sweep_ms = best;
  s->launches = 0;
  check_status(s);
  reset_waves(s);
}

// ---------------------------------------------------------------- port-response form (port.cu)

// S_j = P^T K_j^{-1} P from unit sources at the ports with zero incident waves: 32 port columns
// per launch of the multi-RHS band sweep where it fits in shared memory, else the solver's own
// sweep with its R columns.  Only the subgraphs of the main launch get an S_j: subgraphs flagged
// ill-conditioned keep their FP64 band sweep every sweep (S_j in FP32 would carry the same
// cancellation that made their FP32 factor fail).
template <typename T>
static void compute_port_response(vtm_solver* s, int64_t s_tiles) {
  cudaStream_t st = s->stream;
  const int np = s->npieces;
  s->S.alloc((size_t)s_tiles * kNB * kNB * sizeof(T));
  VTM_CUDA(cudaMemsetAsync(s->S.p, 0, s->S.bytes, st));
  const size_t kSmemMax = 227 * 1024;
  int st_lo = 0;
  size_t sm_lo = 0;
  if (!s->wide && s->cap <= kWideWindow)
    for (int k : {8, 6, 4, 3, 2}) {
      const size_t b = sweep_wide_smem_bytes(sizeof(T), 32, k, s->slot_elems, s->cap);
      if (!st_lo && b <= kSmemMax) st_lo = k, sm_lo = b;
    }
  cudaEvent_t e0, e1;
  VTM_CUDA(cudaEventCreate(&e0));
  VTM_CUDA(cudaEventCreate(&e1));
  VTM_CUDA(cudaEventRecord(e0, st));
  if (st_lo) {
    constexpr int Rs = 32;
    DevBuf bt32, xc32, w0, wsc;
    bt32.alloc((size_t)s->C * Rs * sizeof(T));
    xc32.alloc((size_t)s->C * Rs * sizeof(T));
    w0.alloc((size_t)std::max<int64_t>(1, s->E) * Rs * sizeof(T));
    wsc.alloc(w0.bytes);
    VTM_CUDA(cudaMemsetAsync(w0.p, 0, w0.bytes, st));
    VTM_CUDA((sweep_wide_configure<T, T>(Rs, sm_lo)));
    // the tensor-core form of the multi-RHS sweep where it applies (FP32 band factor, half-bandwidths
    // <= 384), its factor kept only for these solves
    DevBuf wt_tmp;
    if constexpr (sizeof(T) == 4) {
      size_t fb = 0, tb = 0;
      VTM_CUDA(cudaMemGetInfo(&fb, &tb));
      if (s->wt_ok && s->np_lo > 0 && (double)s->wt_bytes < 0.4 * (double)fb) {
        wt_tmp.alloc((size_t)s->wt_bytes);
        VTM_CUDA(cudaMemsetAsync(wt_tmp.p, 0, (size_t)wide_tc_zero_bytes(), st));
        VTM_CUDA(wide_tc_configure(Rs));
        VTM_CUDA(launch_wide_tc_factor(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->wt_max_groups, s->factor.as<float>(),
                                       wt_tmp.as<unsigned char>(), st));
      }
    }
    const int nb = (s->max_ports + Rs - 1) / Rs;
    for (int b = 0; b < nb; ++b) {
      VTM_CUDA(launch_unit_rhs<T>(s->pieces.as<PieceDesc>(), np, s->port_local.as<int32_t>(), Rs, b, bt32.as<T>(), st));
      if (s->np_lo > 0) {
        SweepArgs<T, T> a = sweep_args<T, T>(s, 1, false);
        a.bt = bt32.as<T>();
        a.xc = xc32.as<T>();
        a.wprev = w0.as<T>();
        a.wnext = wsc.as<T>();
        a.stages = st_lo;
        a.withhold = -1;
        a.yspill = nullptr;
        a.cpl.ptr = nullptr;  // unit sources, zero waves: no coupling current
        a.wt = wt_tmp.as<unsigned char>();
        if constexpr (sizeof(T) == 4) {
          if (a.wt) VTM_CUDA(launch_sweep_wide_tc(a, Rs, s->np_lo, st));
          else VTM_CUDA((launch_sweep_wide<T, T>(a, Rs, s->np_lo, sm_lo, st)));
        } else {
          VTM_CUDA((launch_sweep_wide<T, T>(a, Rs, s->np_lo, sm_lo, st)));
        }
      }
      VTM_CUDA(launch_gather_port_response<T>(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->port_local.as<int32_t>(),
                                              Rs, b, xc32.as<T>(), s->S.as<T>(), st));
    }
    VTM_CUDA(cudaStreamSynchronize(st));
  } else {
    const int R = s->R;
    const int nb = (s->max_ports + R - 1) / R;
    for (int b = 0; b < nb; ++b) {
      VTM_CUDA(launch_unit_rhs<T>(s->pieces.as<PieceDesc>(), np, s->port_local.as<int32_t>(), R, b, s->bt.as<T>(), st));
      reset_waves(s);
      sweeps_typed<T>(s, 1);
      if constexpr (sizeof(T) == 4) {
        if (s->port_tc) {
          VTM_CUDA(launch_gather_port_blocks(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->port_local.as<int32_t>(), R, b,
                                             s->xc.as<float>(), s->S.as<float>(), st));
          continue;
        }
      }
      VTM_CUDA(launch_gather_port_response<T>(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->port_local.as<int32_t>(),
                                              R, b, s->xc.as<T>(), s->S.as<T>(), st));
    }
    VTM_CUDA(cudaMemsetAsync(s->bt.p, 0, s->bt.bytes, st));
    reset_waves(s);
  }
  VTM_CUDA(cudaEventRecord(e1, st));
  VTM_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  VTM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->info.port_setup_ms = ms;
  check_status(s);
}

// u_base = P^T K_j^{-1} b̃_j: one band sweep with zero incident waves (its waves go to scratch).
template <typename T>
static void ubase_typed(vtm_solver* s) {
  if (s->np_lo > 0) {
    SweepArgs<T, T> a = sweep_args<T, T>(s, 1, false);
    a.wprev = s->wzero.as<T>();
    a.wnext = s->wscr.as<T>();
    a.cpl.ptr = nullptr;  // zero waves: no coupling current
    launch_one<T, T>(s, a, s->np_lo, s->sweep_smem, s->pipe);
  }
  VTM_CUDA(launch_gather_ports<T>(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->port_local.as<int32_t>(), s->R,
                                  s->xc.as<T>(), s->ubase.as<T>(), s->stream));
  s->launches++;
  s->ubase_ok = true;
}

// Port form, at the start of a defect-correction phase (zero waves): the first sweep of the phase
// is a band sweep from zero incident waves, which is exactly the solve that gives u_base, so it
// serves as both (one sweep fewer than computing u_base separately).
template <typename T>
static void first_sweep_typed(vtm_solver* s) {
  sweeps_typed<T>(s, 1);
  VTM_CUDA(launch_gather_ports<T>(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->port_local.as<int32_t>(), s->R,
                                  s->xc.as<T>(), s->ubase.as<T>(), s->stream));
  s->launches++;
  s->ubase_ok = true;
}

static void ensure_ubase(vtm_solver* s) {
  if (!s->port_form || s->ubase_ok) return;
  if (s->precision == VTM_FP32) ubase_typed<float>(s);
  else ubase_typed<double>(s);
}

template <typename T>
static void launch_port(vtm_solver* s) {
  if constexpr (sizeof(T) == 4) {
    if (s->port_tc) {
      PortTCArgs t;
      t.pieces = s->pieces_lo.as<PieceDesc>();
      t.npieces = s->np_lo;
      t.S16 = s->S16.as<unsigned char>();
      t.sig_s = s->sig16.as<float>();
      t.gscale = s->gscale.as<float>();
      t.scratch = s->tc_scratch.as<unsigned char>();
      t.n4max = s->tc_n4max;
      t.tmem_cols = s->tc_tmem_cols;
      t.ubase = s->ubase.as<float>();
      t.wprev = s->w[s->cur].as<float>();
      t.wnext = s->w[s->cur ^ 1].as<float>();
      t.port_end_ptr = s->port_end_ptr.as<int32_t>();
      t.twin = s->twin.as<int32_t>();
      t.invz = s->invz_t.as<float>();
      t.cpl = couple_ref<float>(s);
      t.prec = s->port_rec.as<int4>();
      t.status = s->status.as<int>();
      t.wait_limit = s->wait_limit;
      VTM_CUDA(launch_port_sweep_tc(t, s->R, !s->port_half, s->tc_grid, s->stream));
      s->launches++;
      return;
    }
  }
  PortArgs<T> a;
  a.det = s->port_det ? 1 : 0;
  a.Sh = s->port_half ? s->Sh.p : nullptr;
  a.scale = s->hscale.as<float>();
  a.pieces = s->pieces_lo.as<PieceDesc>();
  a.S = s->S.as<T>();
  a.ubase = s->ubase.as<T>();
  a.wprev = s->w[s->cur].as<T>();
  a.wnext = s->w[s->cur ^ 1].as<T>();
  a.port_end_ptr = s->port_end_ptr.as<int32_t>();
  a.twin = s->twin.as<int32_t>();
  a.invz = s->invz_t.as<T>();
  a.cpl = couple_ref<T>(s);
  VTM_CUDA(launch_port_sweep<T>(a, s->R, s->np_lo, s->port_smem, s->stream));
  s->launches++;
}

// k sweeps in port form: k - 1 port-only sweeps, then one band sweep that also writes x_j.  The
// flagged subgraphs (FP32 solvers) take their FP64 band sweep in every sweep.
template <typename T>
static void port_sweeps_typed(vtm_solver* s, int k) {
  for (int i = 0; i + 1 < k; ++i) {
    if (s->np_lo > 0) launch_port<T>(s);
    if constexpr (sizeof(T) == 4) {
      if (s->np_hi > 0)
        launch_one<double, float>(s, sweep_args<double, float>(s, 0, true), s->np_hi, s->hi_smem, false);
    }
    s->cur ^= 1;
  }
  if (k > 0) sweeps_typed<T>(s, 1);
}

static int64_t launches_per_batch(const vtm_solver* s, int k) {
  const int64_t band = (s->np_lo > 0) + (s->np_hi > 0);
  if (!s->port_form || k < 2) return (int64_t)k * band;
  const int64_t port = (s->np_lo > 0) + (s->np_hi > 0);
  return (int64_t)(k - 1) * port + band;
}

template <typename T>
static void choose_form(vtm_solver* s, const vtm_setup_opts* o, int64_t s_tiles, int64_t band_elems) {
  s->info.sweep_form = VTM_FORM_BAND;
  if (o->sweep_form == VTM_FORM_BAND || s->E == 0) {
    if (o->sweep_form == VTM_FORM_PORT) fail(VTM_ERR_INVALID, "the port form needs at least one line");
    return;
  }
  const size_t kSmemMax = 227 * 1024;
  // S_j only for the subgraphs of the main launch (flagged ones keep their FP64 band sweep)
  std::vector<PieceDesc> lo;
  lo.reserve(s->np_lo);
  // R >= 16 (FP32): tensor-core sweep over the lower block triangle in 128 x 128 blocks (port_tc.cu);
  // R <= 8: SIMT sweep over 32 x 32 tiles (port.cu)
  const bool tc = s->wide && sizeof(T) == 4;
  s_tiles = 0;
  int64_t h_bytes = 0;
  int max_ports_lo = 0;
  for (size_t j = 0; j < s->pd_host.size(); ++j) {
    if (s->piece_bits[j] == 64 && sizeof(T) == 4) continue;
    PieceDesc d = s->pd_host[j];
    d.s_off = s_tiles;
    d.h_off = h_bytes;
    s_tiles += tc ? port_f32_blocks(d.nports) : port_tiles(d.nports);
    h_bytes += tc ? port_f16_bytes(d.nports) : 0;
    max_ports_lo = std::max(max_ports_lo, d.nports);
    lo.push_back(d);
  }
  // tensor memory holds every 128-port super-row of a subgraph at once: n4 R <= 512 columns
  const int n4max = (max_ports_lo + 127) / 128;
  int tmem_cols = 32;
  while (tmem_cols < n4max * s->R) tmem_cols *= 2;
  const bool tmem_ok = n4max * s->R <= 512 && n4max <= kTcMaxSuper;
  const bool det = !tc && port_sweep_det_fits(sizeof(T), s->R, max_ports_lo);
  const size_t smem = tc ? port_tc_smem_bytes(s->R, true) : port_sweep_smem_bytes(sizeof(T), s->R, max_ports_lo, det);
  // bytes one sweep streams (tensor cores: with the lo half) and the device memory setup needs
  const double s_bytes = tc ? (double)h_bytes : (double)s_tiles * kNB * kNB * sizeof(T);
  const double setup_bytes = tc ? s_bytes + (double)s_tiles * 128.0 * 128.0 * 4.0 : s_bytes;
  const double band_bytes = 2.0 * (double)band_elems * sizeof(T);
  size_t free_b = 0, total_b = 0;
  VTM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const bool shape_ok = tc ? tmem_ok : !s->wide;
  const bool fits = shape_ok && s->np_lo > 0 && smem <= kSmemMax && setup_bytes < 0.5 * (double)free_b;
  if (o->sweep_form == VTM_FORM_PORT && !fits)
    fail(VTM_ERR_INVALID, "the port form needs FP32 or nrhs <= 8, port counts whose response vectors fit in "
                          "shared memory (nrhs <= 8) or in tensor memory (ports x nrhs <= 512 x 128 for nrhs "
                          "16 / 32) and room for the port responses in device memory");
  // AUTO: a batch of m sweeps costs (m - 1) port sweeps plus one band sweep in port form (the
  // multi-RHS band sweep is bound by FP32 arithmetic, so there the tensor-core form always wins)
  const double m = std::max(2, s->check_every);
  if (o->sweep_form == VTM_FORM_AUTO && !(fits && (tc || (m - 1) * s_bytes + band_bytes < m * band_bytes))) return;
  s->port_form = true;
  s->port_tc = tc;
  s->info.sweep_form = VTM_FORM_PORT;
  // largest subgraphs first: the block scheduler starts CTAs in index order, so the smallest ones
  // fill the tail of the launch (all launches over pieces_lo write through global indices only)
  std::stable_sort(lo.begin(), lo.end(), [](const PieceDesc& x, const PieceDesc& y) { return x.nports > y.nports; });
  upload(s->pieces_lo, lo, s->stream);
  s->port_smem = smem;
  if (tc) {
    int dev = 0, nsm = 1;
    VTM_CUDA(cudaGetDevice(&dev));
    VTM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    s->tc_grid = std::min(s->np_lo, nsm);  // one persistent CTA per SM (it holds the SM's tensor memory)
    s->tc_n4max = n4max;
    s->tc_tmem_cols = tmem_cols;
    s->tc_scratch.alloc((size_t)s->tc_grid * ((size_t)2 * n4max * s->R * 512 + (size_t)n4max * 128 * s->R * 4));
    s->S16.alloc((size_t)std::max<int64_t>(1024, h_bytes));
    s->sig16.alloc((size_t)std::max(1, s->np_lo) * sizeof(float));
    s->gscale.alloc((size_t)std::max(1, s->nports) * sizeof(float));
    VTM_CUDA(cudaMemsetAsync(s->gscale.p, 0, s->gscale.bytes, s->stream));
    s->tc_bytes_all = h_bytes;
    s->tc_bytes_hi = h_bytes / 2;
    s->port_rec.alloc((size_t)std::max(1, s->nports) * 3 * sizeof(int4));
    VTM_CUDA(launch_port_records(s->nports, s->port_end_ptr.as<int32_t>(), s->twin.as<int32_t>(),
                                 s->invz_t.as<float>(), couple_ref<float>(s), s->port_rec.as<int4>(), s->stream));
    VTM_CUDA(port_tc_configure(s->R));
  } else {
    VTM_CUDA(port_sweep_configure<T>(s->R, smem, det));
    s->port_det = det;
  }
  s->ubase.alloc((size_t)std::max(1, s->nports) * s->R * sizeof(T));
  s->wzero.alloc((size_t)s->E * s->R * sizeof(T));
  s->wscr.alloc(s->wzero.bytes);
  VTM_CUDA(cudaMemsetAsync(s->wzero.p, 0, s->wzero.bytes, s->stream));
  compute_port_response<T>(s, s_tiles * (tc ? 128 * 128 / (kNB * kNB) : 1));
  s->info.port_bytes = (int64_t)s_bytes;
  s->info.port_storage_bits = 8 * (int)sizeof(T);
  if constexpr (sizeof(T) == 4) {
    // FP16_AUTO only where the sweep streams S_j from HBM: responses that stay in the 126 MB L2
    // gain nothing from half the bytes and would pay the extra sweeps of FP16 rounding
    const bool l2_resident = s_bytes <= 96.0 * (1 << 20);
    if (tc) {
      // fp16 hi / lo blocks of S_j / sigma_j from the FP32 setup blocks, which are then released
      VTM_CUDA(cudaMemsetAsync(s->S16.p, 0, s->S16.bytes, s->stream));
      VTM_CUDA(launch_port_blocks_to_f16(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->S.as<float>(),
                                         s->S16.as<unsigned char>(), s->sig16.as<float>(),
                                         s->gscale.as<float>(), s->stream));
      VTM_CUDA(cudaStreamSynchronize(s->stream));
      s->S.alloc(0);
      // the hi half alone (FP16 storage) only when asked for: with one scale per subgraph its
      // rounding stalls the defect correction of coupled lines (256^3 x 32: 906 sweeps and 8
      // restarts against 482 and 2 with the lo half), so FP16_AUTO keeps the lo half here
      (void)l2_resident;
      if (o->port_storage == VTM_STORE_FP16) {
        s->port_half = true;
        s->info.port_bytes = s->tc_bytes_hi;
        s->info.port_storage_bits = 16;
      }
    }
    if (!tc && (o->port_storage == VTM_STORE_FP16 || (o->port_storage == VTM_STORE_FP16_AUTO && !l2_resident))) {
      s->Sh.alloc((size_t)s_tiles * kNB * kNB * sizeof(__half));
      s->hscale.alloc((size_t)std::max<int64_t>(1, s_tiles) * sizeof(float));  // one scale per tile
      VTM_CUDA(launch_port_to_half(s->pieces_lo.as<PieceDesc>(), s->np_lo, s->S.as<float>(), s->Sh.as<__half>(),
                                   s->hscale.as<float>(), s->stream));
      s->port_half = true;
      s->port_half_auto = (o->port_storage == VTM_STORE_FP16_AUTO);
      s->info.port_bytes = (int64_t)(s_bytes / 2);
      s->info.port_storage_bits = 16;
    }
  }
  // one port sweep, timed
  ensure_ubase(s);
  cudaEvent_t e0, e1;
  VTM_CUDA(cudaEventCreate(&e0));
  VTM_CUDA(cudaEventCreate(&e1));
  port_sweeps_typed<T>(s, 2);
  VTM_CUDA(cudaEventRecord(e0, s->stream));
  for (int i = 0; i < 3; ++i) {
    if (s->np_lo > 0) launch_port<T>(s);
    s->cur ^= 1;
  }
  VTM_CUDA(cudaEventRecord(e1, s->stream));
  VTM_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  VTM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->info.port_sweep_ms = ms / 3;
  s->launches = 0;
  check_status(s);
  reset_waves(s);
}

// Def. 7.1 on the device: g_c = (K_j^{-1})_{cc} for every port copy, nrhs unit right-hand sides
// per subgraph per sweep with zero incident waves (no exchange); the input impedance seen by end e
// (its own line open, every other line terminated) is g_c / (1 - g_c / Z_e) (rank-one downdate).
template <typename T>
static void input_impedances_typed(vtm_solver* s, std::vector<double>& r_api) {
  DevBuf g;
  g.alloc((size_t)std::max(1, s->nports) * sizeof(double));
  const int R = s->R;
  const int nb = (s->max_ports + R - 1) / R;
  for (int b = 0; b < nb; ++b) {
    VTM_CUDA(launch_unit_rhs<T>(s->pieces.as<PieceDesc>(), s->npieces, s->port_local.as<int32_t>(), R, b,
                                s->bt.as<T>(), s->stream));
    reset_waves(s);
    sweeps_typed<T>(s, 1);
    VTM_CUDA(launch_gather_diag<T>(s->pieces.as<PieceDesc>(), s->npieces, s->port_local.as<int32_t>(), R, b,
                                   s->xc.as<T>(), g.as<double>(), s->stream));
  }
  std::vector<double> gh(std::max(1, s->nports));
  VTM_CUDA(cudaMemcpyAsync(gh.data(), g.p, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
  check_status(s);
  r_api.assign(s->E, 0.0);
  for (int64_t k = 0; k < s->E; ++k) {
    const double gc = gh[s->end_port[k]];
    const double z = s->Z[s->end_api[k] >> 1];
    const double den = 1.0 - gc / z;
    // den > 0 in exact arithmetic (the end's own admittance is part of K_j); a port held almost
    // entirely by its line is open-circuit-like: its impedance is capped at 1e12 g_c
    double r = den > 1e-12 ? gc / den : gc * 1e12;
    if (!(r > 0) || !std::isfinite(r)) r = gc > 0 ? gc : z;
    r_api[s->end_api[k]] = r;
  }
  VTM_CUDA(cudaMemsetAsync(s->bt.p, 0, s->bt.bytes, s->stream));
  s->ubase_ok = false;
  reset_waves(s);
}

void solver_input_impedances(vtm_solver* s, double* r) {
  if (!r) fail(VTM_ERR_INVALID, "null output");
  if (s->coupled) fail(VTM_ERR_INVALID, "input impedances (Def. 7.1) are defined here for uncoupled lines only");
  std::vector<double> v;
  if (s->precision == VTM_FP32) input_impedances_typed<float>(s, v);
  else input_impedances_typed<double>(s, v);
  std::copy(v.begin(), v.end(), r);
}

static void run_sweeps_direct(vtm_solver* s, int k) {
  if (s->port_form && k >= 2) {
    if (s->precision == VTM_FP32) port_sweeps_typed<float>(s, k);
    else port_sweeps_typed<double>(s, k);
    return;
  }
  if (s->precision == VTM_FP32) sweeps_typed<float>(s, k);
  else sweeps_typed<double>(s, k);
}

// k sweeps; batches of two or more sweeps replay a captured CUDA graph (one launch instead of k).
// The graph bakes in the buffer pointers, which stay fixed for the solver's lifetime; the wave
// buffer that a batch starts from is part of the key.
void run_sweeps(vtm_solver* s, int k) {
  ensure_ubase(s);
  if (k < 2 || !s->use_graphs) {
    run_sweeps_direct(s, k);
    return;
  }
  for (auto& g : s->graphs)
    if (g.k == k && g.cur == s->cur) {
      VTM_CUDA(cudaGraphLaunch(g.exec, s->stream));
      s->cur = (s->cur + k) & 1;
      s->launches += launches_per_batch(s, k);
      s->have_copies = true;
      return;
    }
  cudaStreamCaptureStatus cs;
  VTM_CUDA(cudaStreamIsCapturing(s->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // the caller is capturing: just record the launches
    run_sweeps_direct(s, k);
    return;
  }
  const int cur0 = s->cur;
  const int64_t l0 = s->launches;
  cudaGraph_t graph;
  VTM_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  try {
    run_sweeps_direct(s, k);
  } catch (...) {
    cudaStreamEndCapture(s->stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  VTM_CUDA(cudaStreamEndCapture(s->stream, &graph));
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  VTM_CUDA(e);
  s->graphs.push_back({k, cur0, exec});
  s->launches = l0;  // the captured launches did not run; count the replay
  s->cur = cur0;
  VTM_CUDA(cudaGraphLaunch(exec, s->stream));
  s->cur = (cur0 + k) & 1;
  s->launches += launches_per_batch(s, k);
  s->have_copies = true;
}

static void drop_graphs(vtm_solver* s) {
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

void reset_waves(vtm_solver* s) {
  for (int b = 0; b < 2; ++b) VTM_CUDA(cudaMemsetAsync(s->w[b].p, 0, s->w[b].bytes, s->stream));
  s->cur = 0;
  s->have_copies = false;
}

static void split_rhs(vtm_solver* s, const double* src, int64_t ld) {
  s->launches++;
  s->ubase_ok = false;
  if (s->precision == VTM_FP32)
    VTM_CUDA(launch_split<float>(s->C, s->R, s->copy_vertex.as<int64_t>(), s->share.as<double>(), src, ld,
                                 s->bt.as<float>(), s->stream));
  else
    VTM_CUDA(launch_split<double>(s->C, s->R, s->copy_vertex.as<int64_t>(), s->share.as<double>(), src, ld,
                                  s->bt.as<double>(), s->stream));
}

static void assemble(vtm_solver* s, const double* xbase, double* xt) {
  s->launches++;
  if (s->precision == VTM_FP32)
    VTM_CUDA(launch_assemble<float>(s->n, s->R, s->vc_ptr.as<int64_t>(), s->vc_copy.as<int64_t>(),
                                    s->xc.as<float>(), xbase, xt, s->n, s->stream));
  else
    VTM_CUDA(launch_assemble<double>(s->n, s->R, s->vc_ptr.as<int64_t>(), s->vc_copy.as<int64_t>(),
                                     s->xc.as<double>(), xbase, xt, s->n, s->stream));
}

vtm_solver* create_solver(const vtm_partition* p, const vtm_setup_opts* o, void* cuda_stream) {
  Range range("vtm_setup");
  auto t0 = std::chrono::steady_clock::now();
  if (!p || !o) fail(VTM_ERR_INVALID, "null partition or options");
  if (o->precision != VTM_FP32 && o->precision != VTM_FP64) fail(VTM_ERR_INVALID, "unknown precision");
  if (!(o->nrhs == 1 || o->nrhs == 2 || o->nrhs == 4 || o->nrhs == 8 || o->nrhs == 16 || o->nrhs == 32))
    fail(VTM_ERR_INVALID, "nrhs must be 1, 2, 4, 8, 16 or 32");
  if (o->z_mode != VTM_Z_UNIFORM && o->z_mode != VTM_Z_EXPLICIT && o->z_mode != VTM_Z_MATCHED &&
      o->z_mode != VTM_Z_LEARNED)
    fail(VTM_ERR_INVALID, "unknown z_mode");
  if (o->z_mode == VTM_Z_LEARNED && !o->model) fail(VTM_ERR_INVALID, "LEARNED z_mode needs a model");
  if (o->z_mode == VTM_Z_EXPLICIT && !o->z_lines && !p->line_a.empty()) fail(VTM_ERR_INVALID, "z_lines is NULL");
  if (o->z_mode == VTM_Z_MATCHED) {
    // §7.1 impedance matching, computed in FP64 (the rank-one downdate of Def. 7.1 cancels badly in
    // FP32 when a line's admittance dominates its port): an FP64 solver with Z = z_uniform on every
    // line gives each end's input impedance, every line takes the geometric mean of its two ends,
    // and the requested solver is built with those impedances.
    vtm_setup_opts t = *o;
    t.precision = VTM_FP64;
    t.z_mode = VTM_Z_UNIFORM;
    t.withhold_slab = 0;
    t.sweep_variant = 0;
    t.sweep_form = VTM_FORM_BAND;
    t.ncouplings = 0;  // matching is done on the uncoupled lines; the couplings are added after
    std::unique_ptr<vtm_solver> tmp;
    for (int r : {8, 4, 2, 1}) {
      t.nrhs = r;
      try {
        tmp.reset(create_solver(p, &t, cuda_stream));
        break;
      } catch (const Error& e) {
        if (e.code != VTM_ERR_INVALID || r == 1) throw;
      }
    }
    std::vector<double> rin;
    input_impedances_typed<double>(tmp.get(), rin);
    tmp.reset();
    const size_t nl = p->line_a.size();
    std::vector<double> Zm(nl);
    for (size_t t2 = 0; t2 < nl; ++t2) Zm[t2] = std::sqrt(rin[2 * t2] * rin[2 * t2 + 1]);
    vtm_setup_opts e = *o;
    e.z_mode = VTM_Z_EXPLICIT;
    e.z_lines = Zm.data();
    vtm_solver* s = create_solver(p, &e, cuda_stream);
    s->info.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return s;
  }
  std::unique_ptr<vtm_solver> s(new vtm_solver());
  s->precision = o->precision;
  s->R = o->nrhs;
  s->check_every = o->check_every > 0 ? o->check_every : 10;
  s->inner_reduction = o->inner_reduction > 0 ? o->inner_reduction : 1e-4;
  if (o->wait_polls < 0) fail(VTM_ERR_INVALID, "wait_polls must be >= 0");
  if (o->sweep_variant < 0 || o->sweep_variant > 3) fail(VTM_ERR_INVALID, "sweep_variant must be 0, 1, 2 or 3");
  if (o->sweep_form < 0 || o->sweep_form > 2) fail(VTM_ERR_INVALID, "sweep_form must be 0, 1 or 2");
  if (o->port_storage < 0 || o->port_storage > 2) fail(VTM_ERR_INVALID, "port_storage must be 0, 1 or 2");
  if (o->wait_polls > 0) s->wait_limit = (long)o->wait_polls;
  if (cuda_stream) {
    s->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    VTM_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  if (s->precision == VTM_FP32) setup_typed<float>(p, o, s.get());
  else setup_typed<double>(p, o, s.get());
  s->info.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return s.release();
}

void solver_set_rhs(vtm_solver* s, const double* b, int64_t ldb) {
  if (!b || ldb < s->n) fail(VTM_ERR_INVALID, "b: null or ldb < n");
  const double* src = b;
  if (!is_device_ptr(b)) {
    for (int r = 0; r < s->R; ++r)
      VTM_CUDA(cudaMemcpyAsync(s->vb.as<double>() + r * s->n, b + r * ldb, s->n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    src = s->vb.as<double>();
    ldb = s->n;
  }
  split_rhs(s, src, ldb);
}

void solver_iterate(vtm_solver* s, int k) {
  Range range("vtm_iterate");
  if (k < 0) fail(VTM_ERR_INVALID, "negative sweep count");
  run_sweeps(s, k);
}

static void read_norms(vtm_solver* s, int cnt) {
  VTM_CUDA(cudaMemcpyAsync(s->h_norms, s->norms.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
}

int solver_solve(vtm_solver* s, const double* b, double* x, int64_t ld, double rtol, int maxit, vtm_stats* stats) {
  Range range("vtm_solve");
  auto t0 = std::chrono::steady_clock::now();
  s->hist_sweeps.clear();
  s->hist_rel.clear();
  s->hist_inner.clear();
  const int64_t launches0 = s->launches;
  if (!b || !x || ld < s->n || !(rtol > 0) || maxit < 1) fail(VTM_ERR_INVALID, "vtm_solve: bad arguments");
  const int R = s->R;
  const int64_t n = s->n;
  const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
  cudaStream_t st = s->stream;
  double* db = s->vb.as<double>();
  if (bdev) {
    VTM_CUDA(launch_copy2d(n, R, b, ld, db, n, st));
    s->launches++;
  } else
    for (int r = 0; r < R; ++r)
      VTM_CUDA(cudaMemcpyAsync(db + r * n, b + r * ld, n * sizeof(double), cudaMemcpyHostToDevice, st));
  double* norms = s->norms.as<double>();
  VTM_CUDA(cudaMemsetAsync(norms, 0, 2 * kMaxRhs * sizeof(double), st));
  VTM_CUDA(cudaMemsetAsync(s->status.p, 0, sizeof(int), st));
  VTM_CUDA(launch_sqnorm_det(n, R, db, n, s->nparts.as<double>(), norms + kMaxRhs, st));
  VTM_CUDA(launch_copy2d(n, R, db, n, s->vr.as<double>(), n, st));
  s->launches += 3;
  read_norms(s, 2 * kMaxRhs);
  std::vector<double> bn(R);
  for (int r = 0; r < R; ++r) bn[r] = s->h_norms[kMaxRhs + r] > 0 ? std::sqrt(s->h_norms[kMaxRhs + r]) : 1.0;

  double* xacc = s->vx.as<double>();   // accepted solution
  double* xt = s->vxt.as<double>();    // trial solution
  double* rcur = s->vr.as<double>();   // residual the current inner solve works on
  double* rt = s->vrt.as<double>();    // trial residual
  VTM_CUDA(cudaMemsetAsync(xacc, 0, n * R * sizeof(double), st));
  std::vector<double> rcur_norm(bn);
  split_rhs(s, rcur, n);
  reset_waves(s);

  const bool refine = (s->precision == VTM_FP32);
  const int m = s->check_every;
  int sweeps = 0, checks = 0, restarts = 0, inner_sweeps = 0;
  double prev_inner = INFINITY, rel = INFINITY;
  int status = VTM_ERR_NOT_CONVERGED;
  bool trial_fresh = false;  // xt holds the assembled iterate of the last check
  // Port form: a batch's last sweep is a band sweep, which costs several port sweeps, so batches are
  // sized from the observed contraction rate to end near the next event (rtol, or the restart
  // threshold of the defect correction), between m and 8 m sweeps.  The rate is measured between
  // two checks of the same inner solve.  A correction phase starts from zero waves and its inner
  // residual first grows (to several times the residual it corrects) before it falls, so its first
  // check comes after 2 m sweeps, and the batch after it is sized from the rate of the phase
  // before (every phase iterates the same operator).
  int next_k = m;
  double last_inner = -1.0;
  int last_inner_sweeps = 0;
  double phase_rate = -1.0;  // per-sweep contraction of the inner residual, last measured
  double phase_rate_before = -1.0;  // phase_rate before its last update
  // port form: the first sweep of every phase also gives u_base (first_sweep_typed)
  auto phase_start = [&]() {
    if (!s->port_form) return;
    if (s->precision == VTM_FP32) first_sweep_typed<float>(s);
    else first_sweep_typed<double>(s);
    ++sweeps;
    ++inner_sweeps;
  };
  phase_start();
  while (sweeps < maxit) {
    const int k = std::min(next_k, maxit - sweeps);
    {
      Range r("vtm_solve/sweeps");
      run_sweeps(s, k);
    }
    sweeps += k;
    inner_sweeps += k;
    assemble(s, xacc, xt);
    VTM_CUDA(launch_residual_det(n, R, s->a_rowptr.as<int64_t>(), s->a_col.as<int32_t>(), s->a_val.as<double>(), db,
                                 n, xt, n, rt, n, s->nparts.as<double>(), norms, st));
    s->launches += 2;
    read_norms(s, R);
    ++checks;
    check_status(s);
    rel = 0;
    double inner = 0;
    bool bad = false;
    for (int r = 0; r < R; ++r) {
      const double rn = std::sqrt(s->h_norms[r]);
      if (!std::isfinite(rn)) bad = true;
      rel = std::max(rel, rn / bn[r]);
      inner = std::max(inner, rn / rcur_norm[r]);
    }
    s->hist_sweeps.push_back(sweeps);
    s->hist_rel.push_back(rel);
    s->hist_inner.push_back(inner);
    if (bad) {
      status = VTM_ERR_DIVERGED;
      break;
    }
    trial_fresh = true;
    if (rel <= rtol) {
      s->vx.swap(s->vxt);
      xacc = s->vx.as<double>();
      status = VTM_OK;
      break;
    }
    next_k = m;
    // sweeps on FP16 port responses stall near the FP16 rounding level of the inner solve, so such a
    // phase restarts once it is within a few units of 2^-11 instead of waiting for the stall
    const double reduction = s->port_half ? std::max(s->inner_reduction, kHalfReduction) : s->inner_reduction;
    double rate = -1.0;
    bool slow = false;  // the inner solve has met its floor
    const int batch = inner_sweeps - last_inner_sweeps;
    if (s->port_form && last_inner > 0 && inner > 0 && batch > 0) {
      const double r_obs = std::pow(inner / last_inner, 1.0 / batch);
      // an interval that gained less than a quarter of what the last healthy one gained per sweep
      // (on the log scale) is a stall
      slow = phase_rate > 0.0 && inner < 1.0 && std::log(r_obs) > 0.25 * std::log(phase_rate);
      if (inner < last_inner) rate = r_obs;
      if (inner <= 0.5 * last_inner) {  // an interval of real progress
        phase_rate_before = phase_rate;
        phase_rate = r_obs;
      }
    } else if (s->port_form && last_inner < 0 && restarts > 0 && inner > 0) {
      rate = phase_rate;  // first check of a correction phase
    }
    if (rate > 0.0 && rate < 1.0) {
      double need = rtol / rel;                                   // reduction to reach rtol
      if (refine) need = std::max(need, reduction / inner);           // or the restart threshold
      if (need < 1.0) {
        const double kk = std::ceil(1.05 * std::log(need) / std::log(rate));
        next_k = (int)std::min<double>(8.0 * m, std::max<double>(m, kk));
      }
    }
    // a correction phase usually ends on its FP32 floor, which only a second check can show: after a
    // long batch in such a phase the next check comes after m / 2 sweeps (at the floor the inner
    // residual moves by about a percent over them, a phase still converging gains a factor of
    // several, so the slow rule tells the two apart)
    if (s->port_form && refine && restarts > 0 && last_inner > 0 && batch > 4 * m) next_k = std::max(2, m / 2);
    last_inner = inner;
    last_inner_sweeps = inner_sweeps;
    // accept the trial only when it improves on the residual it started from
    // FP16 port responses: a correction step that gains less than a factor 10, or an inner solve
    // that has not gained anything after 4 check intervals, means the FP16 rounding is what limits
    // the sweeps; go back to the FP32 responses for the rest of the solver's life
    if (s->port_half && s->port_half_auto &&
        ((inner > 0.1 && inner >= 0.98 * prev_inner && inner_sweeps >= 2 * m) || (inner >= 1.0 && inner_sweeps >= 4 * m))) {
      s->port_half = false;
      s->info.port_storage_bits = 32;
      s->info.port_bytes = s->port_tc ? s->tc_bytes_all : 2 * s->info.port_bytes;
      drop_graphs(s);
    }
    // coupled lines on FP16 responses: while such a phase makes progress it gains far more than a
    // factor 2 per check, so a check that gains less has met the FP16 floor
    const bool half_floor = s->port_half && s->coupled && inner > 0.5 * prev_inner && inner_sweeps >= 2 * m;
    const bool stalled = (inner >= 0.98 * prev_inner && inner_sweeps >= 2 * m) || half_floor || slow;
    if (refine && inner < 1.0 && (inner <= reduction || stalled)) {
      // a phase that ends on a stall spent the end of its last long interval on its floor, so the
      // rate measured over that interval is too slow for sizing the next phase's batches
      if (stalled && inner > reduction && phase_rate_before > 0.0 && phase_rate_before < phase_rate)
        phase_rate = phase_rate_before;
      // defect correction: accept the trial iterate and restart the sweeps on its FP64 residual
      s->vx.swap(s->vxt);
      s->vr.swap(s->vrt);
      xacc = s->vx.as<double>();
      xt = s->vxt.as<double>();
      rcur = s->vr.as<double>();
      rt = s->vrt.as<double>();
      for (int r = 0; r < R; ++r) rcur_norm[r] = std::max(std::sqrt(s->h_norms[r]), 1e-300);
      split_rhs(s, rcur, n);
      reset_waves(s);
      ++restarts;
      inner_sweeps = 0;
      prev_inner = INFINITY;
      last_inner = -1.0;
      next_k = s->port_form ? 2 * m : m;
      trial_fresh = false;
      phase_start();
      continue;
    }
    prev_inner = inner;
  }
  if (status != VTM_OK && trial_fresh) {
    // return the iterate of the last check
    s->vx.swap(s->vxt);
    xacc = s->vx.as<double>();
  }
  if (xdev) {
    VTM_CUDA(launch_copy2d(n, R, xacc, n, x, ld, st));
    s->launches++;
  } else
    for (int r = 0; r < R; ++r)
      VTM_CUDA(cudaMemcpyAsync(x + r * ld, xacc + r * n, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  VTM_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    stats->sweeps = sweeps;
    stats->checks = checks;
    stats->restarts = restarts;
    stats->rel_residual = rel;
    stats->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = (int32_t)(s->launches - launches0);
  }
  if (status == VTM_ERR_NOT_CONVERGED) set_last_error("vtm_solve: maxit reached before rtol");
  if (status == VTM_ERR_DIVERGED) set_last_error("vtm_solve: residual is not finite");
  return status;
}

template <typename T>
static void get_state_typed(vtm_solver* s, double* waves) {
  std::vector<T> h((size_t)s->E * s->R);
  VTM_CUDA(cudaMemcpyAsync(h.data(), s->w[s->cur].p, h.size() * sizeof(T), cudaMemcpyDeviceToHost, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
  for (int64_t e = 0; e < s->E; ++e)
    for (int r = 0; r < s->R; ++r) waves[e + r * s->E] = (double)h[(size_t)s->api_to_int[e] * s->R + r];
}

template <typename T>
static void set_state_typed(vtm_solver* s, const double* waves) {
  std::vector<T> h((size_t)s->E * s->R);
  for (int64_t e = 0; e < s->E; ++e)
    for (int r = 0; r < s->R; ++r) h[(size_t)s->api_to_int[e] * s->R + r] = (T)waves[e + r * s->E];
  VTM_CUDA(cudaMemcpyAsync(s->w[s->cur].p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
}

template <typename T>
static void get_copies_typed(vtm_solver* s, double* out) {
  std::vector<T> h((size_t)s->C * s->R);
  VTM_CUDA(cudaMemcpyAsync(h.data(), s->xc.p, h.size() * sizeof(T), cudaMemcpyDeviceToHost, s->stream));
  VTM_CUDA(cudaStreamSynchronize(s->stream));
  for (int64_t c = 0; c < s->C; ++c)
    for (int r = 0; r < s->R; ++r) out[c + r * s->C] = (double)h[(size_t)c * s->R + r];
}

void solver_get_state(vtm_solver* s, double* waves) {
  if (!waves) fail(VTM_ERR_INVALID, "null waves");
  if (s->precision == VTM_FP32) get_state_typed<float>(s, waves);
  else get_state_typed<double>(s, waves);
}
void solver_set_state(vtm_solver* s, const double* waves) {
  if (!waves) fail(VTM_ERR_INVALID, "null waves");
  if (s->precision == VTM_FP32) set_state_typed<float>(s, waves);
  else set_state_typed<double>(s, waves);
}
void solver_get_copies(vtm_solver* s, double* out) {
  if (!out) fail(VTM_ERR_INVALID, "null output");
  if (!s->have_copies) fail(VTM_ERR_INVALID, "no sweep has run since the last reset");
  if (s->precision == VTM_FP32) get_copies_typed<float>(s, out);
  else get_copies_typed<double>(s, out);
}
void solver_get_info(const vtm_solver* s, vtm_solver_info* info) { *info = s->info; }

void solver_get_history(const vtm_solver* s, int32_t* count, int32_t* sweeps, double* rel, double* inner) {
  *count = (int32_t)s->hist_sweeps.size();
  if (sweeps) std::copy(s->hist_sweeps.begin(), s->hist_sweeps.end(), sweeps);
  if (rel) std::copy(s->hist_rel.begin(), s->hist_rel.end(), rel);
  if (inner) std::copy(s->hist_inner.begin(), s->hist_inner.end(), inner);
}
void solver_get_piece_precision(const vtm_solver* s, int32_t* bits) {
  if (!bits) fail(VTM_ERR_INVALID, "null output");
  std::copy(s->piece_bits.begin(), s->piece_bits.end(), bits);
}
void solver_get_impedances(const vtm_solver* s, double* z) {
  if (!z) fail(VTM_ERR_INVALID, "null output");
  std::copy(s->Z.begin(), s->Z.end(), z);
}
void solver_destroy(vtm_solver* s) { delete s; }

}  // namespace vtm
