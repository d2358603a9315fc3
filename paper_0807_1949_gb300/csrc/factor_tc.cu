// Banded Cholesky of the FP32 local matrices with the trailing update on the tensor cores.
//
// The same blocked right-looking factorisation as factor.cu (kNB = 32 columns per step: factor
// the diagonal block with one warp in shared memory, solve the panel L_IK = A_IK L_KK^{-T} below it,
// update the trailing band, invert the diagonal block), for subgraphs whose half-bandwidth makes
// the update a sizeable dense product: the update A_IJ -= L_IK L_JK^T of the w x w window is a
// symmetric rank-32 product of the panel with itself, issued as tcgen05.mma (kind::tf32, M = 128
// rows per step, N up to 256 columns, K = 8) with both operands read from one K-major copy of the
// panel in shared memory (128-byte swizzle: rows of 32 FP32 entries, 16-byte units XOR-ed with the
// row index mod 8, 8-row groups 1024 bytes apart).  Three TF32 products per term (hi(P) hi(P)^T +
// hi(P) lo(P)^T + lo(P) hi(P)^T, hi = TF32 truncation, lo = the exact FP32 remainder; the split of
// Ootomo and Yokota, 2022) keep the FP32 accuracy of the update; the product accumulates in
// tensor memory and the lower triangle inside the band is subtracted from the band in global
// memory.  One CTA per subgraph, 256 threads; the MMA wait is bounded (status VTM_ERR_TIMEOUT).
#include "kernels.h"

namespace vtm {

namespace {

constexpr int kTB = 128;          // panel rows per MMA (M)
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
  // K-major, 128-byte swizzle, 8-row groups 1024 bytes apart, descriptor version 1
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__host__ __device__ constexpr uint32_t idesc_tf32_kk(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTB >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t swz128(int row, int col) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((col * 4) >> 4) ^ (row & 7)) << 4) + ((col * 4) & 15));
}

__device__ __forceinline__ float hi_tf32(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

}  // namespace

size_t factor_tc_smem_bytes(int max_w) {
  const int mpad = ((max_w + kTB - 1) / kTB) * kTB;
  // barriers | hi(P) | lo(P) | D (32 x 33) | P (max_w x 33) | per-warp 32 x 33 transpose tiles
  return 1024 + 1024 + 2 * (size_t)mpad * 128 + sizeof(float) * 33 * (size_t)(kNB + max_w + 8 * 32);
}

__global__ void __launch_bounds__(256, 1) k_factor_tc(const PieceDesc* __restrict__ pieces, float* band, int* status,
                                                      int* piece_flag, float* diag0, int max_w, long wait_limit) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int bad;   // 1: non-positive pivot, 2: pivot^2 < kFlagRatio * original diagonal
  __shared__ int failed;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  uint64_t* mma_done = reinterpret_cast<uint64_t*>(sm);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 8);
  const int mpad = ((max_w + kTB - 1) / kTB) * kTB;
  const uint32_t phi_s = base + 1024, plo_s = phi_s + (uint32_t)mpad * 128;
  float* phi = reinterpret_cast<float*>(sm + 1024);
  float* plo = reinterpret_cast<float*>(sm + 1024 + mpad * 128);
  float* D = reinterpret_cast<float*>(sm + 1024 + 2 * mpad * 128);
  float* P = D + kNB * 33;                 // panel rows, [max_w][33]
  float* tiles = P + (size_t)max_w * 33;   // [8 warps][32][33]

  const PieceDesc pd = pieces[blockIdx.x];
  float* B = band + pd.factor_off;
  const int Wp = pd.Wp, off = Wp - 1, w = pd.w, n_pad = pd.n_pad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    bad = 0;
    failed = 0;
    mbar_init(mma_done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (diag0)
    for (int r = tid; r < n_pad; r += blockDim.x) diag0[pd.row_off + r] = B[(int64_t)r * Wp + off];
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;

  for (int k0 = 0; k0 < n_pad && !failed; k0 += kNB) {
    // (a) diagonal block of the updated band
    for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
      const int r = idx / kNB, c = idx % kNB;
      D[r * 33 + c] = (c <= r) ? B[(int64_t)(k0 + r) * Wp + off - (r - c)] : 0.f;
    }
    __syncthreads();
    // (b) its Cholesky factor, by warp 0
    if (warp == 0) {
      // right-looking Cholesky of the block in shared memory, lane i owning row i: at step j lane j
      // takes the pivot, the lanes below scale their entry of column j and update their row
      const float d0 = diag0 ? diag0[pd.row_off + k0 + lane] : D[lane * 33 + lane];
      for (int j = 0; j < kNB; ++j) {
        if (lane == j) {
          float djj = D[j * 33 + j];
          if (!(djj > 0.f)) {
            bad = 1;
            djj = 1.f;
          } else if (djj < (float)kFlagRatio * d0 && bad == 0) {
            bad = 2;
          }
          D[j * 33 + j] = sqrtf(djj);
        }
        __syncwarp();
        if (lane > j) D[lane * 33 + j] /= D[j * 33 + j];
        __syncwarp();
        if (lane > j) {
          const float lij = D[lane * 33 + j];
          for (int c = j + 1; c <= lane; ++c) D[lane * 33 + c] -= lij * D[c * 33 + j];
        }
        __syncwarp();
      }
      for (int c = lane + 1; c < kNB; ++c) D[lane * 33 + c] = 0.f;
    }
    __syncthreads();
    // (c) panel rows below the block within the band, L_IK = A_IK L_KK^{-T}; the K-major hi / lo
    // copies for the tensor cores
    int nrows = n_pad - k0 - kNB;
    if (nrows > w) nrows = w;
    if (nrows < 0) nrows = 0;
    // panel block in, coalesced: row ri, column c at band position off - (ri + kNB - c)
    for (int idx = tid; idx < nrows * kNB; idx += blockDim.x) {
      const int ri = idx / kNB, c = idx % kNB;
      const int dist = ri + kNB - c;
      P[ri * 33 + c] = (dist <= off) ? B[(int64_t)(k0 + kNB + ri) * Wp + off - dist] : 0.f;
    }
    __syncthreads();
    for (int ri = tid; ri < nrows; ri += blockDim.x) {
      float x[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c) x[c] = P[ri * 33 + c];
#pragma unroll
      for (int c = 0; c < kNB; ++c) {
        float s = x[c];
#pragma unroll
        for (int k = 0; k < c; ++k) s -= x[k] * D[c * 33 + k];
        x[c] = s / D[c * 33 + c];
      }
#pragma unroll
      for (int c = 0; c < kNB; ++c) {
        P[ri * 33 + c] = x[c];
        const float h = hi_tf32(x[c]);
        phi[swz128(ri, c) / 4] = h;
        plo[swz128(ri, c) / 4] = x[c] - h;
      }
    }
    __syncthreads();
    // panel block out, coalesced
    for (int idx = tid; idx < nrows * kNB; idx += blockDim.x) {
      const int ri = idx / kNB, c = idx % kNB;
      const int dist = ri + kNB - c;
      if (dist <= off) B[(int64_t)(k0 + kNB + ri) * Wp + off - dist] = P[ri * 33 + c];
    }
    fence_proxy_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // (d) trailing update A_IJ -= L_IK L_JK^T, j <= i, inside the band: 128 panel rows at a time
    for (int I0 = 0; I0 < nrows && !failed; I0 += kTB) {
      const int ncols = (nrows < I0 + kTB ? nrows : I0 + kTB);  // columns j < ncols can meet rows of this step
      const int nr = ((ncols + 15) / 16) * 16;
      if (tid == 0) {
        for (int n0 = 0; n0 < nr; n0 += 256) {
          const int nn = (nr - n0 < 256) ? nr - n0 : 256;
          const uint32_t idesc = idesc_tf32_kk(nn);
#pragma unroll
          for (int kk = 0; kk < kNB / 8; ++kk) {
            const uint64_t aH = sdesc_k(phi_s + (uint32_t)I0 * 128 + kk * 32);
            const uint64_t aL = sdesc_k(plo_s + (uint32_t)I0 * 128 + kk * 32);
            const uint64_t bH = sdesc_k(phi_s + (uint32_t)n0 * 128 + kk * 32);
            const uint64_t bL = sdesc_k(plo_s + (uint32_t)n0 * 128 + kk * 32);
            mma_tf32(tmem + n0, aH, bH, idesc, kk > 0 ? 1u : 0u);
            mma_tf32(tmem + n0, aH, bL, idesc, 1u);
            mma_tf32(tmem + n0, aL, bH, idesc, 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mma_done))
                     : "memory");
      }
      if (!mbar_wait_bounded(mma_done, phase, wait_limit)) {
        failed = 1;
        // the MMAs complete in any case; they must before tensor memory is freed
        mbar_wait_bounded(mma_done, phase, kDrainPolls);
      }
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      __syncthreads();  // every thread now sees the same `failed`
      if (!failed) {
        // warp q = warp % 4 reads lanes 32 q .. + 31 (rows I0 + 32 q + lane); warps 0-3 take the even
        // 32-column chunks, warps 4-7 the odd ones
        const int q = warp & 3;
        const int i = I0 + q * 32 + lane;
        const int imin = I0 + q * 32, imax = imin + 31;
        for (int c0 = (warp >> 2) * 32; c0 < nr; c0 += 64) {
          if (c0 > imax || imin - (c0 + 31) > off) continue;  // no j <= i inside the band here
          uint32_t v[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
              : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0)
              : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          // turn the 32 x 32 block around through shared memory (lane = row -> lane = column), so
          // that each update of a band row is one coalesced run of 32 entries
          float* tile = tiles + warp * (32 * 33);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) tile[lane * 33 + jj] = __uint_as_float(v[jj]);
          __syncwarp();
          const int j = c0 + lane;
          float cur[32];
#pragma unroll
          for (int ii = 0; ii < 32; ++ii) {
            const int ir = imin + ii;
            cur[ii] = (ir < nrows && j <= ir && ir - j <= off) ? B[(int64_t)(k0 + kNB + ir) * Wp + off - ir + j] : 0.f;
          }
#pragma unroll
          for (int ii = 0; ii < 32; ++ii) {
            const int ir = imin + ii;
            if (ir < nrows && j <= ir && ir - j <= off)
              B[(int64_t)(k0 + kNB + ir) * Wp + off - ir + j] = cur[ii] - tile[ii * 33 + lane];
          }
          __syncwarp();
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // (e) replace the diagonal block by inv(L_KK) (column j by thread j)
    if (tid < kNB) {
      const int j = tid;
      float X[kNB];
#pragma unroll
      for (int i = 0; i < kNB; ++i) {
        if (i < j) {
          X[i] = 0.f;
        } else if (i == j) {
          X[i] = 1.f / D[i * 33 + i];
        } else {
          float s = 0.f;
#pragma unroll
          for (int k = 0; k < i; ++k)
            if (k >= j) s += D[i * 33 + k] * X[k];
          X[i] = -s / D[i * 33 + i];
        }
      }
#pragma unroll
      for (int i = 0; i < kNB; ++i)
        if (i >= j) B[(int64_t)(k0 + i) * Wp + off - (i - j)] = X[i];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (failed) atomicExch(status, kStatusTimeout);
    if (bad) {
      if (piece_flag) piece_flag[blockIdx.x] = bad;
      else if (bad == 1) atomicExch(status, kStatusNotSpd);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

cudaError_t launch_factor_tc(const PieceDesc* pieces, int npieces, int max_w, float* band, int* status,
                             int* piece_flag, float* diag0, long wait_limit, cudaStream_t st) {
  const size_t smem = factor_tc_smem_bytes(max_w);
  if (smem > 227 * 1024 || max_w > 3 * kTB) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_factor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (npieces > 0) k_factor_tc<<<npieces, 256, smem, st>>>(pieces, band, status, piece_flag, diag0, max_w, wait_limit);
  return cudaGetLastError();
}

}  // namespace vtm
