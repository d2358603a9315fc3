// Device-side layout shared by the CUDA kernels of libvtm (sm_103a).
//
// Band storage of a subgraph's factor (eq. 5.8, factored once, §8): n_pad rows (n_j rounded up to
// kNB with identity rows), each row Wp entries, RIGHT-aligned so that entry p of row i holds
// column i - (Wp-1) + p (p = Wp-1 is the diagonal).  Columns left of the band (or negative) hold
// zeros.  After the factorisation every kNB x kNB diagonal block holds the INVERSE of the
// Cholesky block L_KK (lower triangular), so the substitution is matrix-vector work only.
// Wp >= kNB so that a full diagonal block always fits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vtm {

constexpr int kNB = 32;            // rows per block (slab) of the substitution and factorisation
constexpr int kSweepThreads = 256; // 8 threads per slab row
constexpr int kMaxStages = 16;     // slab ring depth limit (the 128-byte mbarrier area holds 16)

// Polls allowed when a CTA that gave up drains the bulk copies it has issued (they target valid
// memory and complete; the limit only keeps the drain bounded).
constexpr long kDrainPolls = 1L << 26;

// Status word written by kernels (0 = ok); values are vtm_status codes.
constexpr int kStatusNotSpd = 4;
constexpr int kStatusTimeout = 7;

// A subgraph whose FP32 Cholesky pivot keeps less than this fraction of its original diagonal
// (pivot^2 / K_ii < kFlagRatio: the matrix is close to singular for FP32) is refactored in FP64.
constexpr double kFlagRatio = 1e-5;

struct PieceDesc {
  int64_t factor_off;  // element offset of row 0 of this piece's band
  int64_t copy_off;    // first copy (global copy id) of the piece
  int32_t n;           // local unknowns n_j
  int32_t n_pad;       // n_j rounded up to kNB
  int32_t Wp;          // stored row width (>= w_j + 1, >= kNB)
  int32_t w;           // half-bandwidth w_j
  int32_t port_off;    // first port (index into port arrays)
  int32_t nports;
  int32_t end_off;     // first (sorted) line end of the piece
  int32_t nends;
  int64_t row_off;     // first padded row of the piece in per-row arrays (sum of earlier n_pad)
  int64_t s_off;       // first 32 x 32 tile (port.cu) or 128 x 128 FP32 setup block (port_tc.cu) of S_j
  int64_t h_off;       // port_tc.cu: byte offset of the piece's fp16 port-response blocks
  int64_t wt_off;      // sweep_wide_tc.cu: byte offset of the piece's tensor-core factor groups
};

// ------------------------------------------------------------------ PTX wrappers (sm_90+)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Adds `bytes` to the transaction count of the current phase without arriving: a phase fed by
// several copies issued at different times completes once the one arrival has come and all of
// their bytes have landed.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared (TMA engine), completion counted on `bar` in bytes.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of an mbarrier phase (cheaper than try_wait when the phase is already complete).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (each poll may suspend the
// thread for a hardware-defined slice), returning false so that the caller can record a timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long limit) {
  if (mbar_test_wait(bar, parity)) return true;  // already complete: no suspend
  for (long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <typename T>
__device__ __forceinline__ T warp_sum_g8(T v) {
  // sum over the 8 consecutive lanes of a group (lane bits 0..2)
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

// Coupled lines (§7.2): the bundle admittance Y = diag(1/Z_t) + sum_p y_p (e_t - e_t')(e_t - e_t')^T.
// Its diagonal (1/Z_t + sum of the line's y_p) is the per-end 1/Z array that every sweep kernel
// already applies to the end's own incoming wave; the off-diagonal part adds, at the port of end e
// of line t, -y_p w_in[e'] for every pair (t, t'), e' the end of t' at the same subgraph.  Stored
// per port (CSR over all ports): for entry k, oth[k] indexes the incoming wave w_in[e'] (the twin
// of e') and y[k] = -y_p.
template <typename TV>
struct CoupleRef {
  const int32_t* ptr;  // nports_total + 1 entry offsets; nullptr: uncoupled lines
  const int32_t* oth;
  const TV* y;
};

template <typename T, typename TV>
__device__ __forceinline__ T coupling_current(const CoupleRef<TV>& c, int port, int r, int R, const TV* w) {
  T acc = T(0);
  for (int k = c.ptr[port]; k < c.ptr[port + 1]; ++k) acc += (T)c.y[k] * (T)w[(size_t)c.oth[k] * R + r];
  return acc;
}

}  // namespace vtm
