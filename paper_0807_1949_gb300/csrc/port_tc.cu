// Port-response sweep for 16 or 32 right-hand sides on the 5th-generation tensor cores.
//
// Per subgraph the sweep needs y = S_j s (then u = u_base + y, w_out = 2u - w_in; see port.cu for
// the method).  With R = 16/32 columns this is a dense matrix product, so it runs as tcgen05.mma
// (kind::tf32, FP32 accumulation in tensor memory), both operands K-major:
//
//  * S_j is stored whole (both triangles) as 128 x 32 chunks (I, c): ports 128 I .. 128 I + 127
//    by ports 32 c .. 32 c + 31, in the 128-byte-swizzled K-major layout the tensor core reads
//    (rows of 128 bytes, 16-byte units XOR-ed with the row index mod 8, 8-row groups 1024 bytes
//    apart), chunks of a row of super-blocks contiguous.  A symmetric half would need the transposed
//    operand (MN-major), which this build does not use for TF32.
//  * s^T (32 columns x ports, zero beyond R and beyond the port count) is written by the CTA to a
//    global scratch in the same layout, 4 KB per 32 ports (B operand, K-major).
//  * Chunk (I, c) adds S_Ic s_c to y_I: four MMAs of K = 8.  y lives in tensor memory: 128 lanes
//    (one port each) x 32 columns per super-row, up to 16 super-rows (2048 ports) in 512 columns.
//
// One CTA per subgraph, 256 threads.  Thread 0 issues the bulk copies of a stage ring (S chunk +
// s chunk = 20 KB per stage, mbarrier complete_tx) and the MMAs; tcgen05.commit frees a stage once
// its MMAs have read it.  Every wait is bounded; a CTA that gives up records VTM_ERR_TIMEOUT, lets
// its copies and MMAs finish, frees its tensor memory and returns.
#include "kernels.h"

namespace vtm {

namespace {

constexpr int kTB = 128;                        // ports per super-row (MMA M)
constexpr int kTN = 32;                         // accumulator columns per super-row (MMA N)
constexpr int kKC = 32;                         // ports per K chunk
constexpr uint32_t kChunkBytes = kTB * kKC * 4; // S chunk: 128 x 32 FP32
constexpr uint32_t kVecBytes = kTN * kKC * 4;   // s chunk: 32 columns x 32 ports
constexpr uint32_t kStageBytes = kChunkBytes + kVecBytes;
constexpr int kTcStages = 6;
constexpr int kTcThreads = 256;

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Shared-memory matrix descriptor: start address, leading / stride byte offsets (16-byte units),
// descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor, kind::tf32: FP32 accumulator, A and B TF32, M = 128, N = 32; a_mn / b_mn
// select MN-major operands.
__host__ __device__ constexpr uint32_t idesc_tf32(bool a_mn, bool b_mn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTB >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// FP32 -> TF32 with round-to-nearest (ties away), kept in a 32-bit container; the tensor core
// ignores the low 13 mantissa bits, so rounding here halves the operand error of truncation.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of (row, 4-byte column) inside a 128-byte-swizzled block of 128-byte rows.
__host__ __device__ __forceinline__ uint32_t swz(int row, int col) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((col * 4) >> 4) ^ (row & 7)) << 4) + ((col * 4) & 15));
}

}  // namespace

int64_t port_blocks_tc(int nports) {
  const int64_t n4 = (nports + kTB - 1) / kTB, nkc = (nports + kKC - 1) / kKC;
  return n4 * nkc;
}

int64_t port_vec_chunks_tc(int nports) { return (nports + kKC - 1) / kKC; }

size_t port_tc_smem_bytes() { return 1024 + 1024 + (size_t)kTcStages * kStageBytes; }

// S_j columns cc = b * Rs + r from unit-source solves into the chunk layout (whole matrix).
__global__ void k_gather_port_response_tc(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local,
                                          int Rs, int b, const float* __restrict__ xc, float* __restrict__ S) {
  const PieceDesc pd = pieces[blockIdx.x];
  const int nkc = (pd.nports + kKC - 1) / kKC;
  for (int i = threadIdx.x; i < pd.nports * Rs; i += blockDim.x) {
    const int q = i / Rs, r = i % Rs;
    const int cc = b * Rs + r;
    if (cc >= pd.nports) continue;
    const int64_t chunk = pd.s_off + (int64_t)(q / kTB) * nkc + cc / kKC;
    S[chunk * (kChunkBytes / 4) + swz(q % kTB, cc % kKC) / 4] =
        to_tf32(xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * Rs + r]);
  }
}

template <int R>
__global__ void __launch_bounds__(kTcThreads, 1) k_port_sweep_tc(const PortTCArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int abort_flag;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);  // [kTcStages]
  uint64_t* empty = full + kTcStages;                // [kTcStages]
  uint64_t* done = empty + kTcStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const uint32_t stage0 = base + 1024;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int np = pd.nports;
  if (np == 0) return;
  const int n4 = (np + kTB - 1) / kTB;
  const int nkc = (np + kKC - 1) / kKC;
  const int nchunk = n4 * nkc;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // s^T: sum_e w_in[e] / Z_e per port and column, rounded to TF32, zero padding; row = column r
  // of the right-hand side, 128 bytes = 32 ports per chunk
  float* sg = a.sglob + pd.v_off * (kVecBytes / 4);
  for (int i = tid; i < nkc * kKC * kTN; i += kTcThreads) {
    const int r = i / (nkc * kKC), p = i % (nkc * kKC);
    float v = 0.f;
    if (p < np && r < R) {
      const int e0 = a.port_end_ptr[pd.port_off + p], e1 = a.port_end_ptr[pd.port_off + p + 1];
      for (int e = e0; e < e1; ++e) v += a.wprev[(size_t)a.twin[e] * R + r] * a.invz[e];
    }
    sg[(p / kKC) * (kVecBytes / 4) + swz(r, p % kKC) / 4] = to_tf32(v);
  }
  asm volatile("fence.proxy.async;" ::: "memory");  // generic-proxy writes -> bulk-copy reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (tid == 0) {
    const float* Sp = a.S + pd.s_off * (kChunkBytes / 4);
    int issued = 0;
    auto load = [&](int st) {
      const uint32_t sb = stage0 + st * kStageBytes;
      mbar_arrive_expect_tx(&full[st], kStageBytes);
      bulk_g2s(sb, Sp + (int64_t)issued * (kChunkBytes / 4), kChunkBytes, &full[st]);
      bulk_g2s(sb + kChunkBytes, sg + (issued % nkc) * (kVecBytes / 4), kVecBytes, &full[st]);
      ++issued;
    };
    for (int st = 0; st < kTcStages && st < nchunk; ++st) load(st);
    constexpr uint32_t kId = idesc_tf32(false, false);  // A = S chunk, B = s^T chunk, both K-major
    int b = 0;
    for (; b < nchunk; ++b) {
      const int st = b % kTcStages;
      const uint32_t ph = (uint32_t)((b / kTcStages) & 1);
      if (!mbar_wait_bounded(&full[st], ph, a.wait_limit)) {
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int I = b / nkc, c = b % nkc;
      const uint32_t sb = stage0 + st * kStageBytes;
#pragma unroll
      for (int kk = 0; kk < kKC / 8; ++kk)
        mma_tf32(tmem + I * kTN, sdesc(sb + kk * 32, 16, 1024), sdesc(sb + kChunkBytes + kk * 32, 16, 1024), kId,
                 (c > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[st]);
      if (issued < nchunk) {
        if (!mbar_wait_bounded(&empty[st], ph, a.wait_limit)) {
          abort_flag = 1;
          ++b;
          break;
        }
        load(st);
      }
    }
    if (abort_flag) {
      // let the copies already issued land before the shared memory goes away
      for (int b2 = b; b2 < issued; ++b2)
        mbar_wait_bounded(&full[b2 % kTcStages], (uint32_t)((b2 / kTcStages) & 1), kDrainPolls);
      atomicExch(a.status, kStatusTimeout);
    }
    mma_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(done, 0, kDrainPolls) && !abort_flag;
  tc_fence_after();

  if (ok) {
    // u = u_base + y; w_out[e] = 2 u - w_in[e].  Warp w reads lanes 32 (w % 4) .. + 31 of every
    // other super-row.
    const int q = warp & 3;
    for (int bb = warp >> 2; bb < n4; bb += 2) {
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(bb * kTN), v);
      const int p = bb * kTB + q * 32 + lane;
      if (p < np) {
        const float* ub = a.ubase + (size_t)(pd.port_off + p) * R;
        const int e0 = a.port_end_ptr[pd.port_off + p], e1 = a.port_end_ptr[pd.port_off + p + 1];
        for (int e = e0; e < e1; ++e) {
          const float* wi = a.wprev + (size_t)a.twin[e] * R;
          float* wo = a.wnext + (size_t)e * R;
#pragma unroll
          for (int r = 0; r < R; ++r) wo[r] = 2.f * (ub[r] + __uint_as_float(v[r])) - wi[r];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tmem_cols)
                 : "memory");
  }
}

cudaError_t port_tc_configure(int R) {
  const int smem = (int)port_tc_smem_bytes();
  switch (R) {
    case 16: return cudaFuncSetAttribute(k_port_sweep_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case 32: return cudaFuncSetAttribute(k_port_sweep_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_port_sweep_tc(const PortTCArgs& a, int R, int npieces, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  const size_t smem = port_tc_smem_bytes();
  switch (R) {
    case 16: k_port_sweep_tc<16><<<npieces, kTcThreads, smem, st>>>(a); break;
    case 32: k_port_sweep_tc<32><<<npieces, kTcThreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_port_response_tc(const PieceDesc* pieces, int npieces, const int32_t* port_local, int Rs,
                                           int b, const float* xc, float* S, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_gather_port_response_tc<<<npieces, 256, 0, st>>>(pieces, port_local, Rs, b, xc, S);
  return cudaGetLastError();
}

}  // namespace vtm
