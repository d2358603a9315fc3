// Host-callable launchers of the libvtm CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <cuda_fp16.h>

#include "device.cuh"

namespace vtm {

// Arguments of one VTM sweep (Table 1 steps 3-5) over a set of subgraphs.  TF: factor and
// substitution type; TV: type of the sources, local solutions, waves and 1/Z in global memory.
template <typename TF, typename TV = TF>
struct SweepArgs {
  const PieceDesc* pieces;     // the subgraphs of this launch, one CTA each
  const TF* factor;            // band factors (see device.cuh)
  const TF* factor_u;          // transposed band (rows of U = L^T, left-aligned), R <= 8 kernel
  const TV* bt;                // b̃: copies x R, R contiguous
  TV* xc;                      // local solutions: copies x R (written when write_x)
  const TV* wprev;             // outgoing waves of the previous sweep: ends x R
  TV* wnext;                   // outgoing waves of this sweep
  const int32_t* port_local;   // per port: local row of the port copy
  const int32_t* port_end_ptr; // per port: first (sorted) end; nports_total + 1 entries
  const int32_t* twin;         // per end: the twin end of the same line
  const TV* invz;              // per end: 1 / Z_e
  int* status;                 // kernel status word (0 = ok)
  int write_x;
  int stages;                  // staged slabs in flight (>= 2)
  int slot_elems;              // ring slot stride in elements (kNB * max Wp)
  int ys_elems;                // (2 (max Wp - 1) + max n_pad) * R
  int win_elems;               // (max ends per piece) * R
  long wait_limit;             // bounded mbarrier polls before a timeout is recorded
  int withhold;                // testing: slab index whose copy is never issued (-1 = none)
  int cap;                     // wide kernel: window rows (power of two >= max Wp - 1 + kNB)
  TF* yspill;                  // wide kernel: forward result y in factor precision, n_pad x R per
                               // piece at row_off (nullptr: y goes through xc, TF == TV)
  CoupleRef<TV> cpl;           // coupled lines: per-port coupling lists (cpl.ptr == nullptr: none)
  const unsigned char* wt;     // tensor-core factor of sweep_wide_tc.cu (nullptr: not built)
};

size_t sweep_smem_bytes(size_t elem, int R, int stages, int slot_elems, int ys_elems, int win_elems);
template <typename TF, typename TV>
cudaError_t sweep_configure(int R, size_t smem);
template <typename TF, typename TV>
cudaError_t sweep_occupancy(int R, size_t smem, int* ctas_per_sm);
template <typename TF, typename TV>
cudaError_t launch_sweep(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st);

// Pipelined variant (R = 1, 2): warp 0 finishes block k while warps 1-7 prepare block k+1.
size_t sweep_pipe_smem_bytes(size_t elem, int R, int stages, int slot_elems, int ys_elems, int win_elems);
template <typename TF, typename TV>
cudaError_t sweep_pipe_configure(int R, size_t smem);
template <typename TF, typename TV>
cudaError_t sweep_pipe_occupancy(int R, size_t smem, int* ctas_per_sm);
template <typename TF, typename TV>
cudaError_t launch_sweep_pipe(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st);

// Multi-RHS sweep with the band products on the tensor cores (R = 16, 32; FP32 solvers): the factor
// of each subgraph, balanced and split into fp16 hi / lo panels of 128-row groups, built once from
// the FP32 band factor (sweep_wide_tc.cu).  Half-bandwidths up to 128 kWideTcMaxTiles.
constexpr int kWideTcMaxTiles = 3;
int64_t wide_tc_bytes(int n, int w);
int64_t wide_tc_zero_bytes();  // the zero panel the factor buffer starts with
bool wide_tc_fits(int w);
int wide_tc_groups(int n);
size_t wide_tc_smem_bytes(int R);
cudaError_t wide_tc_configure(int R);
cudaError_t launch_wide_tc_factor(const PieceDesc* pieces, int npieces, int max_groups, const float* band,
                                  unsigned char* wt, cudaStream_t st);
cudaError_t launch_sweep_wide_tc(const SweepArgs<float, float>& a, int R, int npieces, cudaStream_t st);

// Wide variant (R = 16, 32): vectors spill to xc, a circular window of 512 rows stays in shared memory.
size_t sweep_wide_smem_bytes(size_t elem, int R, int stages, int slot_elems, int cap);
template <typename TF, typename TV>
cudaError_t sweep_wide_configure(int R, size_t smem);
template <typename TF, typename TV>
cudaError_t launch_sweep_wide(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st);
// Arguments of one sweep in port-response form (port.cu): u = u_base + S_j s per subgraph.
template <typename T>
struct PortArgs {
  const PieceDesc* pieces;     // all subgraphs, one CTA each
  const T* S;                  // port responses, lower block triangle of 32 x 32 tiles
  const void* Sh;              // FP32 solvers: the same tiles in IEEE half (nullptr: use S)
  const float* scale;          // FP16 storage: per stored tile (global tile index), the factor it was divided by
  const T* ubase;              // P^T K_j^{-1} b̃_j: ports x R
  const T* wprev;              // outgoing waves of the previous sweep: ends x R
  T* wnext;                    // outgoing waves of this sweep
  const int32_t* port_end_ptr;
  const int32_t* twin;
  const T* invz;
  CoupleRef<T> cpl;            // coupled lines (cpl.ptr == nullptr: none)
  int det;                     // per-warp column accumulators summed in a fixed order (bitwise
                               // reproducible); 0: shared-memory atomics
};

// Shared memory the deterministic SIMT port sweep may take (it keeps three CTAs per SM with FP16
// storage).
constexpr size_t kPortDetSmem = 72 * 1024;

__host__ __device__ int64_t port_tiles(int nports);
size_t port_sweep_smem_bytes(size_t elem, int R, int max_ports, bool det);
bool port_sweep_det_fits(size_t elem, int R, int max_ports);
template <typename T>
cudaError_t port_sweep_configure(int R, size_t smem, bool det);
template <typename T>
cudaError_t launch_port_sweep(const PortArgs<T>& a, int R, int npieces, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_gather_port_response(const PieceDesc* pieces, int npieces, const int32_t* port_local, int Rs, int b,
                                        const T* xc, T* S, cudaStream_t st);
template <typename T>
cudaError_t launch_gather_ports(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, const T* xc,
                                T* ubase, cudaStream_t st);
// FP16 copy (and per-tile scale) of the FP32 port-response tiles.
cudaError_t launch_port_to_half(const PieceDesc* pieces, int npieces, const float* S, __half* Sh, float* scale,
                                cudaStream_t st);

// Tensor-core port-response sweep for 16 / 32 right-hand sides (port_tc.cu), FP32 solvers.
struct PortTCArgs {
  const PieceDesc* pieces;     // subgraphs of the launch (largest first); CTA c takes c, c + grid, ...
  int npieces;
  const unsigned char* S16;    // lower block triangle of S_j / sigma_j as fp16 hi / lo panels (h_off)
  const float* sig_s;          // sigma_j per subgraph of the launch
  const float* gscale;         // g_p = sqrt(S_pp) per port (diagonal balance of S_j)
  unsigned char* scratch;      // per CTA two slots of n4max s^T tiles (R x 512 bytes each)
  int n4max;                   // most 128-port super-rows of a subgraph
  int tmem_cols;               // tensor-memory columns per CTA (power of two >= n4max R)
  const float* ubase;          // ports x R
  const float* wprev;          // ends x R
  float* wnext;
  const int32_t* port_end_ptr;
  const int32_t* twin;
  const float* invz;
  CoupleRef<float> cpl;        // coupled lines (cpl.ptr == nullptr: none)
  const int4* prec;            // per port 3 x int4: first four entries' wave rows, their coefficients
                               // (float bits), {next end, e1, next coupling, k1} (launch_port_records)
  int* status;
  long wait_limit;
};

constexpr int kTcMaxSuper = 16;       // 128-port super-rows per subgraph on the tensor cores
int64_t port_f16_bytes(int nports);   // fp16 hi / lo blocks of one subgraph (1 KB multiple)
int64_t port_f32_blocks(int nports);  // 128 x 128 FP32 blocks of the lower triangle (setup)
size_t port_tc_smem_bytes(int R, bool lo);
// Per-port gather records of the tensor-core port sweep (3 int4 per port, nports of them).
cudaError_t launch_port_records(int nports, const int32_t* port_end_ptr, const int32_t* twin, const float* invz,
                                CoupleRef<float> cpl, int4* rec, cudaStream_t st);
cudaError_t port_tc_configure(int R);
// One persistent launch per sweep (grid <= SMs); lo = use the lo half of S_j (FP32-accurate).
cudaError_t launch_port_sweep_tc(const PortTCArgs& a, int R, bool lo, int grid, cudaStream_t st);
cudaError_t launch_gather_port_blocks(const PieceDesc* pieces, int npieces, const int32_t* port_local, int Rs, int b,
                                      const float* xc, float* S32, cudaStream_t st);
cudaError_t launch_port_blocks_to_f16(const PieceDesc* pieces, int npieces, const float* S32, unsigned char* S16,
                                      float* sig, float* gscale, cudaStream_t st);

constexpr int kWideWindow = 512;
constexpr int kMaxRhs = 32;

// Assemble K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T into the (zeroed) band storage (eq. 5.8).
template <typename T>
cudaError_t launch_build_band(int64_t ncopies, const int32_t* copy_piece, const PieceDesc* pieces,
                              const int64_t* l_rowptr, const int32_t* l_col, const double* l_val,
                              const int32_t* port_of_copy, const int32_t* port_end_ptr, const double* invz,
                              int npieces, int max_pad_rows, T* band, int* status, cudaStream_t st);
// U = L^T (left-aligned rows, transposed inverse diagonal blocks) for the dot-form back substitution.
template <typename T>
cudaError_t launch_transpose_band(const PieceDesc* pieces, int npieces, const T* L, T* U, cudaStream_t st);
// Banded Cholesky of every K_j in place; each diagonal block replaced by its inverse.
// piece_flag[j] (may be NULL): 1 = non-positive pivot, 2 = pivot^2 < kFlagRatio K_ii (precision
// lost); the global status gets kStatusNotSpd only when piece_flag is NULL.  diag0 (may be NULL):
// per-row scratch (sum of n_pad entries) holding the original diagonal.
// FP32 factorisation with the trailing update on the tensor cores (factor_tc.cu), 64 <= max_w <= 384.
size_t factor_tc_smem_bytes(int max_w);
cudaError_t launch_factor_tc(const PieceDesc* pieces, int npieces, int max_w, float* band, int* status,
                             int* piece_flag, float* diag0, long wait_limit, cudaStream_t st);
template <typename T>
cudaError_t launch_factor(const PieceDesc* pieces, int npieces, int max_w, T* band, int* status, int* piece_flag,
                          T* diag0, cudaStream_t st);

// Unit right-hand sides for batch b of every subgraph's ports (b̃ of port b*R + r = e_c in column r).
template <typename T>
cudaError_t launch_unit_rhs(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, int b, T* bt,
                            cudaStream_t st);
// g[port] = x_c of column r for the ports of batch b (diagonal of K_j^{-1}).
template <typename T>
cudaError_t launch_gather_diag(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, int b,
                               const T* xc, double* g, cudaStream_t st);
// b̃_c = share_c * src[vertex(c)]  (§4 step 3), into T precision, R contiguous.
template <typename T>
cudaError_t launch_split(int64_t ncopies, int R, const int64_t* copy_vertex, const double* share,
                         const double* src, int64_t ld, T* bt, cudaStream_t st);
// xt[i] = xbase[i] + mean over the copies of i of xc (xbase may be NULL).
template <typename T>
cudaError_t launch_assemble(int64_t n, int R, const int64_t* vc_ptr, const int64_t* vc_copy, const T* xc,
                            const double* xbase, double* xt, int64_t ld, cudaStream_t st);
// res = b - A x (res may be NULL); norms[r] += ||res_r||^2.
cudaError_t launch_residual(int64_t n, int R, const int64_t* rowptr, const int32_t* col, const double* val,
                            const double* b, int64_t ldb, const double* x, int64_t ldx, double* res, int64_t ldr,
                            double* norms, cudaStream_t st);
// norms[r] += ||v_r||^2
cudaError_t launch_sqnorm(int64_t n, int R, const double* v, int64_t ld, double* norms, cudaStream_t st);
// The same two with fixed-order sums (identical inputs give identical norms): norms[r] = ||res_r||^2
// (resp. ||v_r||^2), through the scratch part of norm_parts(n) * R doubles.
int64_t norm_parts(int64_t n);
cudaError_t launch_residual_det(int64_t n, int R, const int64_t* rowptr, const int32_t* col, const double* val,
                                const double* b, int64_t ldb, const double* x, int64_t ldx, double* res, int64_t ldr,
                                double* part, double* norms, cudaStream_t st);
cudaError_t launch_sqnorm_det(int64_t n, int R, const double* v, int64_t ld, double* part, double* norms,
                              cudaStream_t st);
// dst[i + r*ldd] = src[i + r*lds]
cudaError_t launch_copy2d(int64_t n, int R, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st);

}  // namespace vtm
