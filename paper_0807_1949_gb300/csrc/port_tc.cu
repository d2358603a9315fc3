// Port-response sweep for 16 or 32 right-hand sides on the 5th-generation tensor cores.
//
// Per subgraph the sweep needs y = S_j s (then u = u_base + y, w_out = 2u - w_in; see port.cu for
// the method).  With R = 16/32 columns this is a dense matrix product, so it runs as tcgen05.mma
// (kind::tf32, FP32 accumulation in tensor memory), both operands K-major:
//
//  * S_j is stored whole (both triangles, FP32) as 128 x 32 chunks (I, c): ports 128 I .. 128 I +
//    127 by ports 32 c .. 32 c + 31, in the 128-byte-swizzled K-major layout the tensor core reads
//    (rows of 128 bytes, 16-byte units XOR-ed with the row index mod 8, 8-row groups 1024 bytes
//    apart), the chunks of a row of super-blocks contiguous.  A symmetric half would need the
//    transposed operand (MN-major), which this build does not use for TF32.
//  * Three TF32 products keep FP32 accuracy (the split of Ootomo and Yokota, "Recovering single
//    precision accuracy from Tensor Cores while surpassing the FP32 theoretical peak performance",
//    2022): with hi(x) the TF32 truncation of x and lo(x) = x - hi(x) (exact in FP32),
//    S s ~ hi(S) hi(s) + hi(S) lo(s) + lo(S) hi(s).  hi(S) is what the tensor core reads from the
//    FP32 chunk itself; lo(S) is formed in shared memory by six converter warps; hi(s) and lo(s)
//    are written by the CTA to a global scratch (sᵀ: 32 columns x ports, zero padding), 2 x 4 KB
//    per 32 ports.  The dropped lo(S) lo(s) term and the TF32 truncation of the lo parts are
//    below 2^-21 relative to |S||s|.
//  * Chunk (I, c) adds S_Ic s_c to y_I: 3 x 4 MMAs of M = 128, N = 32, K = 8.  y lives in tensor
//    memory: 128 lanes (one port each) x 32 columns per super-row, up to 16 super-rows (2048
//    ports) in 512 columns.
//
// Two launches per sweep.  k_port_vec_tc (one CTA per subgraph) writes hi(s) and lo(s).  Then
// k_port_sweep_tc works on items (subgraph, 128-port super-row I), 256 threads, two CTAs per SM,
// warp-specialised over a 3-stage bulk-copy ring (S chunk + hi(s) + lo(s) = 24 KB) and a 2-buffer
// lo(S) ring: warp 0 issues the bulk copies (mbarrier complete_tx), warps 2-7 form lo(S), warp 1
// issues the MMAs into 32 tensor-memory columns and releases stages and lo buffers with
// tcgen05.commit; then every warp reads its quarter of the 128 lanes and half of the columns and
// writes the waves.  Every wait is bounded; a CTA that gives up records VTM_ERR_TIMEOUT, lets its
// copies and MMAs finish, frees its tensor memory and returns.
#include "kernels.h"

namespace vtm {

namespace {

constexpr int kTB = 128;                        // ports per super-row (MMA M)
constexpr int kTN = 32;                         // accumulator columns per super-row (MMA N)
constexpr int kKC = 32;                         // ports per K chunk
constexpr uint32_t kChunkBytes = kTB * kKC * 4; // S chunk: 128 x 32 FP32
constexpr uint32_t kVecBytes = kTN * kKC * 4;   // s chunk: 32 columns x 32 ports
// bulk-copy stage: S chunk | hi(s) | lo(s); lo(S) goes to a separate ring of kLoBufs buffers
constexpr uint32_t kStageBytes = kChunkBytes + 2 * kVecBytes;
constexpr int kTcStages = 3;
constexpr int kLoBufs = 2;
constexpr uint32_t kTmemCols = 32;              // one super-row of accumulators per CTA
constexpr int kTcThreads = 256;
constexpr int kConvWarps = 6;                   // warps 2..7
constexpr uint32_t kHiMask = 0xFFFFE000u;       // TF32: sign, exponent, 10 mantissa bits

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

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & kHiMask); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

int64_t port_vec_chunks_tc(int nports) { return 2 * ((nports + kKC - 1) / kKC); }

size_t port_tc_smem_bytes() { return 1024 + 1024 + (size_t)kTcStages * kStageBytes + (size_t)kLoBufs * kChunkBytes; }

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
        xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * Rs + r];
  }
}

// hi(s), lo(s) per subgraph: s = sum_e w_in[e] / Z_e per port and column as sᵀ chunks (row =
// column r of the right-hand side, 128 bytes = 32 ports), zero padding.  Warp w takes chunks w,
// w + 8, ...; lane = port of the chunk, so each store of a column writes one 128-byte row and
// the R wave loads of a lane are independent.
template <int R>
__global__ void __launch_bounds__(kTcThreads) k_port_vec_tc(const PortTCArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int np = pd.nports;
  const int nkc = (np + kKC - 1) / kKC;
  float* sg = a.sglob + pd.v_off * (kVecBytes / 4);
  for (int c = warp; c < nkc; c += kTcThreads / 32) {
    const int p = c * kKC + lane;
    int e0 = 0, e1 = 0, tw = 0;
    float iz = 0.f;
    if (p < np) {
      e0 = a.port_end_ptr[pd.port_off + p];
      e1 = a.port_end_ptr[pd.port_off + p + 1];
      tw = a.twin[e0];
      iz = a.invz[e0];
    }
    float v[kTN];
    const float4* w0 = reinterpret_cast<const float4*>(a.wprev + (size_t)tw * R);
#pragma unroll
    for (int k = 0; k < R / 4; ++k) {
      const float4 x = (e1 > e0) ? w0[k] : make_float4(0.f, 0.f, 0.f, 0.f);
      v[4 * k] = x.x * iz;
      v[4 * k + 1] = x.y * iz;
      v[4 * k + 2] = x.z * iz;
      v[4 * k + 3] = x.w * iz;
    }
#pragma unroll
    for (int r = R; r < kTN; ++r) v[r] = 0.f;
    for (int e = e0 + 1; e < e1; ++e) {
      const float* we = a.wprev + (size_t)a.twin[e] * R;
      const float ize = a.invz[e];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] += we[r] * ize;
    }
    if (a.cpl.ptr && p < np)
      for (int k = a.cpl.ptr[pd.port_off + p]; k < a.cpl.ptr[pd.port_off + p + 1]; ++k) {
        const float yk = a.cpl.y[k];
        const float4* wt = reinterpret_cast<const float4*>(a.wprev + (size_t)a.cpl.oth[k] * R);
#pragma unroll
        for (int kk = 0; kk < R / 4; ++kk) {
          const float4 x = wt[kk];
          v[4 * kk] += yk * x.x;
          v[4 * kk + 1] += yk * x.y;
          v[4 * kk + 2] += yk * x.z;
          v[4 * kk + 3] += yk * x.w;
        }
      }
    float* hi_c = sg + (size_t)(2 * c) * (kVecBytes / 4);
    float* lo_c = hi_c + kVecBytes / 4;
#pragma unroll
    for (int r = 0; r < kTN; ++r) {
      const float hi = tf32_hi(v[r]);
      hi_c[swz(r, lane) / 4] = hi;
      lo_c[swz(r, lane) / 4] = v[r] - hi;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kTcThreads, 2) k_port_sweep_tc(const PortTCArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ volatile int abort_flag;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm);  // [kTcStages] bulk copies landed
  uint64_t* empty = full + kTcStages;                // [kTcStages] MMAs done reading the stage
  uint64_t* conv = empty + kTcStages;                // [kLoBufs] lo(S) written
  uint64_t* lofree = conv + kLoBufs;                 // [kLoBufs] MMAs done reading lo(S)
  uint64_t* done = lofree + kLoBufs;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const uint32_t stage0 = base + 1024;
  const uint32_t lo0 = stage0 + kTcStages * kStageBytes;
  unsigned char* stage0_ptr = sm + 1024;
  unsigned char* lo0_ptr = stage0_ptr + kTcStages * kStageBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int2 item = a.items[blockIdx.x];
  const PieceDesc pd = a.pieces[item.x];
  const int I = item.y;
  const int np = pd.nports;
  const int nkc = (np + kKC - 1) / kKC;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kLoBufs; ++s) {
      mbar_init(&conv[s], kConvWarps);
      mbar_init(&lofree[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const float* sg = a.sglob + pd.v_off * (kVecBytes / 4);

  if (warp == 0) {
    // ---- producer: chunk c of super-row I and its port-vector chunk c
    if (lane == 0) {
      const float* Sp = a.S + (pd.s_off + (int64_t)I * nkc) * (kChunkBytes / 4);
      int c = 0;
      for (; c < nkc && !abort_flag; ++c) {
        const int st = c % kTcStages;
        if (c >= kTcStages &&
            !mbar_wait_bounded(&empty[st], (uint32_t)(((c / kTcStages) - 1) & 1), a.wait_limit)) {
          abort_flag = 1;
          break;
        }
        const uint32_t sb = stage0 + st * kStageBytes;
        mbar_arrive_expect_tx(&full[st], kStageBytes);
        bulk_g2s(sb, Sp + (int64_t)c * (kChunkBytes / 4), kChunkBytes, &full[st]);
        bulk_g2s(sb + kChunkBytes, sg + (size_t)(2 * c) * (kVecBytes / 4), 2 * kVecBytes, &full[st]);
      }
      // the copies of the last stages must land before the shared memory can go away
      for (int c2 = (c > kTcStages ? c - kTcStages : 0); c2 < c; ++c2)
        mbar_wait_bounded(&full[c2 % kTcStages], (uint32_t)((c2 / kTcStages) & 1), kDrainPolls);
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      constexpr uint32_t kId = idesc_tf32(false, false);  // both operands K-major
      for (int c = 0; c < nkc; ++c) {
        const int st = c % kTcStages, lb = c % kLoBufs;
        // conv[lb] for chunk c implies full[st] (the converters waited for it)
        if (abort_flag || !mbar_wait_bounded(&conv[lb], (uint32_t)((c / kLoBufs) & 1), a.wait_limit)) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sb = stage0 + st * kStageBytes;
        const uint32_t sS = sb, sL = lo0 + lb * kChunkBytes, vH = sb + kChunkBytes, vL = vH + kVecBytes;
#pragma unroll
        for (int kk = 0; kk < kKC / 8; ++kk) {
          const uint64_t aH = sdesc(sS + kk * 32, 16, 1024), aL = sdesc(sL + kk * 32, 16, 1024);
          const uint64_t bH = sdesc(vH + kk * 32, 16, 1024), bL = sdesc(vL + kk * 32, 16, 1024);
          mma_tf32(tmem, aH, bH, kId, (c > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, aH, bL, kId, 1u);
          mma_tf32(tmem, aL, bH, kId, 1u);
        }
        mma_commit(&empty[st]);
        mma_commit(&lofree[lb]);
      }
      mma_commit(done);  // arrives once every MMA issued above has completed
    }
  } else {
    // ---- converters: lo(S) = S - hi(S) into the lo ring
    const int ct = tid - 64;
    for (int c = 0; c < nkc; ++c) {
      const int st = c % kTcStages, lb = c % kLoBufs;
      if (abort_flag || !mbar_wait_bounded(&full[st], (uint32_t)((c / kTcStages) & 1), a.wait_limit) ||
          (c >= kLoBufs &&
           !mbar_wait_bounded(&lofree[lb], (uint32_t)(((c / kLoBufs) - 1) & 1), a.wait_limit))) {
        abort_flag = 1;
        break;
      }
      const float4* src = reinterpret_cast<const float4*>(stage0_ptr + st * kStageBytes);
      float4* dst = reinterpret_cast<float4*>(lo0_ptr + lb * kChunkBytes);
      for (int i = ct; i < (int)(kChunkBytes / 16); i += 32 * kConvWarps) {
        const float4 x = src[i];
        dst[i] = make_float4(x.x - tf32_hi(x.x), x.y - tf32_hi(x.y), x.z - tf32_hi(x.z), x.w - tf32_hi(x.w));
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[lb]);
    }
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(done, 0, kDrainPolls) && !abort_flag;
  if (abort_flag && tid == 0) atomicExch(a.status, kStatusTimeout);
  tc_fence_after();

  if (ok) {
    // u = u_base + y; w_out[e] = 2 u - w_in[e].  Warp w reads lanes 32 (w % 4) .. + 31 (one port
    // per lane) and the 16 columns 16 (w / 4) .. + 15; rows move as 16-byte vectors.
    const int q = warp & 3, h = warp >> 2;
    if (16 * h < R) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * h))
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int p = I * kTB + q * 32 + lane;
      if (p < np) {
        const float4* ub = reinterpret_cast<const float4*>(a.ubase + (size_t)(pd.port_off + p) * R + 16 * h);
        const int e0 = a.port_end_ptr[pd.port_off + p], e1 = a.port_end_ptr[pd.port_off + p + 1];
        float4 u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float4 b4 = ub[k];
          u[k] = make_float4(b4.x + __uint_as_float(v[4 * k]), b4.y + __uint_as_float(v[4 * k + 1]),
                             b4.z + __uint_as_float(v[4 * k + 2]), b4.w + __uint_as_float(v[4 * k + 3]));
        }
        for (int e = e0; e < e1; ++e) {
          const float4* wi = reinterpret_cast<const float4*>(a.wprev + (size_t)a.twin[e] * R + 16 * h);
          float4* wo = reinterpret_cast<float4*>(a.wnext + (size_t)e * R + 16 * h);
          float4 w[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) w[k] = wi[k];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            wo[k] = make_float4(2.f * u[k].x - w[k].x, 2.f * u[k].y - w[k].y, 2.f * u[k].z - w[k].z,
                                2.f * u[k].w - w[k].w);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
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

cudaError_t launch_port_sweep_tc(const PortTCArgs& a, int R, int npieces, int nitems, cudaStream_t st) {
  if (npieces <= 0 || nitems <= 0) return cudaSuccess;
  const size_t smem = port_tc_smem_bytes();
  switch (R) {
    case 16:
      k_port_vec_tc<16><<<npieces, kTcThreads, 0, st>>>(a);
      k_port_sweep_tc<16><<<nitems, kTcThreads, smem, st>>>(a);
      break;
    case 32:
      k_port_vec_tc<32><<<npieces, kTcThreads, 0, st>>>(a);
      k_port_sweep_tc<32><<<nitems, kTcThreads, smem, st>>>(a);
      break;
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
