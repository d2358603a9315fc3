// One VTM sweep for many right-hand sides at once (R = 16 or 32): the factor of every subgraph is
// streamed once per sweep for all R columns (Table 1 steps 3-5, eq. 5.6 / 5.8 per column).
//
// The subgraph's vectors no longer fit in shared memory, so the CTA keeps a circular window of
// the last Wp-1+32 rows x R in shared memory; the forward pass spills each finished block of y to
// the copies buffer (xc; a factor-precision spill buffer when the vectors are narrower than the
// factor) and the backward pass reads y back and overwrites it with x.  Per 32-row
// block (the window holds `cap` rows, a power of two >= Wp - 1 + 32) the dot part of the forward pass, t = r - L_off y_window, and the column update of the
// backward pass, y_window -= L_off^T x_B, are small dense products done with register tiles of
// 4 rows x 4 columns per thread (the K dimension split across thread groups, partial tiles summed
// in shared memory).  The factor slabs arrive through the same TMA bulk-copy ring as in sweep.cu.
#include "kernels.h"

namespace vtm {

namespace {

// Threads of the multi-RHS kernel: one CTA per SM fits (the slab ring and the vector window fill
// the shared memory), so it carries 16 warps to hide the latency of each block step.
constexpr int kWideThreads = 512;

template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
  } else {
    const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
    v[0] = x.x, v[1] = x.y, v[2] = y.x, v[3] = y.y;
  }
}

template <typename T, int R>
struct WideLayout {
  static constexpr int kRG = kNB / 4;           // row groups (rows rg, rg+8, rg+16, rg+24)
  static constexpr int kCG = R / 4;             // column groups of 4
  static constexpr int kTiles = kRG * kCG;      // thread tiles per block product
  static constexpr int kKS = kWideThreads / kTiles;  // K splits
  static_assert(kKS >= 1 && kWideThreads % kTiles == 0, "tile mapping");
};

}  // namespace

size_t sweep_wide_smem_bytes(size_t elem, int R, int stages, int slot_elems, int cap) {
  const int tiles = (kNB / 4) * (R / 4);
  const int ks = kWideThreads / tiles;
  return 128 + elem * ((size_t)stages * slot_elems + (size_t)cap * R + (size_t)ks * kNB * R + 2 * (size_t)kNB * R);
}

template <typename T, typename TV, int R>
__global__ void __launch_bounds__(kWideThreads, 1) k_sweep_wide(const SweepArgs<T, TV> a) {
  using LY = WideLayout<T, R>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int S = a.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  T* ring = reinterpret_cast<T*>(smem + 128);
  const int kCap = a.cap;
  T* Yw = ring + (size_t)S * a.slot_elems;  // [cap][R]
  T* part = Yw + (size_t)kCap * R;          // [kKS][kNB][R]
  T* TB = part + (size_t)LY::kKS * kNB * R; // [kNB][R]
  T* XB = TB + (size_t)kNB * R;             // [kNB][R]
  const int kMask = kCap - 1;

  const int Wp = pd.Wp;
  const int off = Wp - 1;
  const int nblk = pd.n_pad / kNB;
  const int total = 2 * nblk;
  const uint32_t slab_bytes = (uint32_t)(kNB * Wp * sizeof(T));
  const T* fbase = a.factor + pd.factor_off;
  TV* xg = a.xc + (size_t)pd.copy_off * R;        // y, then x, of this subgraph (n rows x R)
  T* yg = a.yspill ? a.yspill + (size_t)pd.row_off * R : nullptr;  // y in factor precision
  const TV* bg = a.bt + (size_t)pd.copy_off * R;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
    fence_proxy_async_smem();
  }
  __syncthreads();
  auto issue = [&](int s) {
    if (s == a.withhold) return;  // testing hook: this slab's wait can only run out
    const int kb = s < nblk ? s : total - 1 - s;
    const int slot = s % S;
    mbar_arrive_expect_tx(&bars[slot], slab_bytes);
    bulk_copy_g2s(ring + (size_t)slot * a.slot_elems, fbase + (size_t)kb * kNB * Wp, slab_bytes, &bars[slot]);
  };
  if (tid == 0)
    for (int s = 0; s < S && s < total; ++s) issue(s);
  for (int i = tid; i < kCap * R; i += kWideThreads) Yw[i] = T(0);
  __syncthreads();

  // thread tile of the block products
  const int ks = tid / LY::kTiles;
  const int tt = tid % LY::kTiles;
  const int rg = tt / LY::kCG, cg = tt % LY::kCG;

  // r = b̃ + P (Y w_in) for every row of the subgraph first (the port currents gathered from the
  // twins' waves by all threads at once), into the y storage, which the forward pass then reads
  // row block by row block and overwrites with y.
  if (yg) {
    for (int i = tid; i < pd.n * R; i += kWideThreads) yg[i] = (T)bg[i];
  } else {
    for (int i = tid; i < pd.n * R; i += kWideThreads) xg[i] = bg[i];
  }
  __syncthreads();
  for (int i = tid; i < pd.nports * R; i += kWideThreads) {
    const int q = i / R, c = i % R;
    T acc = T(0);
    for (int e = a.port_end_ptr[pd.port_off + q]; e < a.port_end_ptr[pd.port_off + q + 1]; ++e)
      acc += (T)a.wprev[(size_t)a.twin[e] * R + c] * (T)a.invz[e];
    if (a.cpl.ptr) acc += coupling_current<T, TV>(a.cpl, pd.port_off + q, c, R, a.wprev);
    const size_t at = (size_t)a.port_local[pd.port_off + q] * R + c;
    if (yg) yg[at] += acc;
    else xg[at] = (TV)((T)xg[at] + acc);
  }
  __syncthreads();

  // The inputs of a block step are loaded one step ahead into registers, so that their global
  // latency overlaps the block products of the step before: forward, the rows k0 .. k0 + 31 of r;
  // backward, the stored y of the rows k0 - off .. k0 - off + 31.
  constexpr int kPer = kNB * R / kWideThreads;  // elements of a 32-row block per thread
  static_assert(kPer >= 1 && (kNB * R) % kWideThreads == 0, "block elements per thread");
  T in_v[kPer];
  auto prefetch = [&](int s2) {
    if (s2 >= total) return;
    const bool f2 = s2 < nblk;
    const int k2 = (f2 ? s2 : total - 1 - s2) * kNB;
    if (f2) {
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * kWideThreads;
        const int row = k2 + i / R;
        in_v[j] = row < pd.n ? (yg ? yg[(size_t)row * R + i % R] : (T)xg[(size_t)row * R + i % R]) : T(0);
      }
    } else if (s2 > nblk) {
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * kWideThreads;
        const int row = k2 - off + i / R, c = i % R;
        in_v[j] = row >= 0 ? (yg ? yg[(size_t)row * R + c] : (T)xg[(size_t)row * R + c]) : T(0);
      }
    }
  };
  prefetch(0);

  int s = 0;
  for (; s < total; ++s) {
    const bool fwd = s < nblk;
    const int k0 = (fwd ? s : total - 1 - s) * kNB;
    if (fwd) {
      // rows k0..k0+31 of r enter the window
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * kWideThreads;
        Yw[(size_t)((k0 + i / R) & kMask) * R + i % R] = in_v[j];
      }
    } else if (s > nblk) {
      // backward: rows k0 - off .. k0 - off + 31 enter the window from the stored y
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * kWideThreads;
        const int row = k0 - off + i / R;
        if (row >= 0) Yw[(size_t)(row & kMask) * R + i % R] = in_v[j];
      }
    }
    prefetch(s + 1);
    const int slot = s % S;
    if (!mbar_wait_bounded(&bars[slot], (uint32_t)((s / S) & 1), a.wait_limit)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    const T* L = ring + (size_t)slot * a.slot_elems;
    if (fwd) {
      // partial t over this thread's K range of window columns q in [0, off): column k0 - off + q
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
      const int q0 = (off * ks) / LY::kKS, q1 = (off * (ks + 1)) / LY::kKS;
      // columns q < 31 lie left of the band start of some rows (entry q - r < 0): only there the
      // rows need a test
      const int qs = min(q1, max(q0, kNB - 1));
      for (int q = q0; q < qs; ++q) {
        T yv[4];
        load4(Yw + (size_t)((k0 - off + q) & kMask) * R + 4 * cg, yv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = rg + 8 * i;
          const T l = (q >= r) ? L[r * Wp + q - r] : T(0);
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += l * yv[j];
        }
      }
      const T* Lrow = L + rg * (Wp - 1);
#pragma unroll 2
      for (int q = qs; q < q1; ++q) {
        T yv[4];
        load4(Yw + (size_t)((k0 - off + q) & kMask) * R + 4 * cg, yv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T l = Lrow[8 * i * (Wp - 1) + q];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] += l * yv[j];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[((size_t)ks * kNB + rg + 8 * i) * R + 4 * cg + j] = acc[i][j];
      __syncthreads();
      for (int i = tid; i < kNB * R; i += kWideThreads) {
        const int r = i / R, c = i % R;
        T v = Yw[(size_t)((k0 + r) & kMask) * R + c];
#pragma unroll
        for (int k = 0; k < LY::kKS; ++k) v -= part[((size_t)k * kNB + r) * R + c];
        TB[i] = v;
      }
      __syncthreads();
      // y_B = inv(L_KK) t; a thread takes rows r and 31 - r (r + 1 and 32 - r terms: balanced)
      for (int i = tid; i < kNB * R / 2; i += kWideThreads) {
        const int rr[2] = {i / R, kNB - 1 - i / R};
        const int c = i % R;
        T v[2] = {T(0), T(0)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const T* Lr = L + rr[h] * Wp + off - rr[h];
          for (int c2 = 0; c2 <= rr[h]; ++c2) v[h] += Lr[c2] * TB[c2 * R + c];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = rr[h];
          Yw[(size_t)((k0 + r) & kMask) * R + c] = v[h];
          if (k0 + r < pd.n) {
            if (yg) yg[(size_t)(k0 + r) * R + c] = v[h];
            else xg[(size_t)(k0 + r) * R + c] = (TV)v[h];
          }
        }
      }
    } else {
      // x_B = inv(L_KK)^T y_B; rows r and 31 - r per thread (32 - r and r + 1 terms)
      for (int i = tid; i < kNB * R / 2; i += kWideThreads) {
        const int rr[2] = {i / R, kNB - 1 - i / R};
        const int c = i % R;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = rr[h];
          T v = T(0);
          for (int r2 = r; r2 < kNB; ++r2) v += L[r2 * Wp + off - r2 + r] * Yw[(size_t)((k0 + r2) & kMask) * R + c];
          XB[r * R + c] = v;
        }
      }
      __syncthreads();
      for (int i = tid; i < kNB * R; i += kWideThreads) {
        const int r = i / R, c = i % R;
        if (k0 + r < pd.n) xg[(size_t)(k0 + r) * R + c] = (TV)XB[i];
        Yw[(size_t)((k0 + r) & kMask) * R + c] = XB[i];
      }
      // window rows q in [0, off) (column k0 - off + q) -= sum_r L[r][q - r] x_B[r]
      // tiles of 4 consecutive q x 4 columns, split over the threads
      constexpr int kQT = 4;
      const int nq = (off + kQT - 1) / kQT;
      for (int tile = tid; tile < nq * LY::kCG; tile += kWideThreads) {
        const int qb = (tile / LY::kCG) * kQT, cc = (tile % LY::kCG) * 4;
        T acc[kQT][4];
#pragma unroll
        for (int i = 0; i < kQT; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        const int rmax = min(kNB - 1, qb + kQT - 1);
        if (qb >= kNB - 1 && qb + kQT <= off) {
          // every entry q - r of the tile lies inside the band row: no tests
          for (int r = 0; r <= rmax; ++r) {
            T xv[4];
            load4(XB + r * R + cc, xv);
            const T* Lr = L + r * (Wp - 1) + qb;
#pragma unroll
            for (int i = 0; i < kQT; ++i) {
              const T l = Lr[i];
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[i][j] += l * xv[j];
            }
          }
        } else {
          for (int r = 0; r <= rmax; ++r) {
            T xv[4];
            load4(XB + r * R + cc, xv);
#pragma unroll
            for (int i = 0; i < kQT; ++i) {
              const int q = qb + i;
              const T l = (q >= r && q < off) ? L[r * Wp + q - r] : T(0);
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[i][j] += l * xv[j];
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
          const int q = qb + i;
          if (q < off && k0 - off + q >= 0)
#pragma unroll
            for (int j = 0; j < 4; ++j) Yw[(size_t)((k0 - off + q) & kMask) * R + cc + j] -= acc[i][j];
        }
      }
    }
    __syncthreads();
    if (tid == 0 && s + S < total) {
      fence_proxy_async_smem();
      issue(s + S);
    }
  }
  if (abort_flag) {
    if (tid == 0) {
      atomicExch(a.status, kStatusTimeout);
      for (int s2 = s; s2 < total && s2 < s + S; ++s2)
        if (s2 != a.withhold) mbar_wait_bounded(&bars[s2 % S], (uint32_t)((s2 / S) & 1), kDrainPolls);
    }
    return;
  }
  __syncthreads();
  // w_out[e] = 2 x_c - w_in[e]
  for (int i = tid; i < pd.nports * R; i += kWideThreads) {
    const int q = i / R, c = i % R;
    const int l = a.port_local[pd.port_off + q];
    const T x = (T)xg[(size_t)l * R + c];
    for (int e = a.port_end_ptr[pd.port_off + q]; e < a.port_end_ptr[pd.port_off + q + 1]; ++e)
      a.wnext[(size_t)e * R + c] = (TV)(T(2) * x - (T)a.wprev[(size_t)a.twin[e] * R + c]);
  }
}

template <typename TF, typename TV, int R>
static cudaError_t wide_configure_one(size_t smem) {
  return cudaFuncSetAttribute(k_sweep_wide<TF, TV, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename TF, typename TV>
cudaError_t sweep_wide_configure(int R, size_t smem) {
  switch (R) {
    case 16: return wide_configure_one<TF, TV, 16>(smem);
    case 32: return wide_configure_one<TF, TV, 32>(smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TV>
cudaError_t launch_sweep_wide(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  dim3 grid(npieces), block(kWideThreads);
  switch (R) {
    case 16: k_sweep_wide<TF, TV, 16><<<grid, block, smem, st>>>(a); break;
    case 32: k_sweep_wide<TF, TV, 32><<<grid, block, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define VTM_WIDE_INST(TF, TV)                                  \
  template cudaError_t sweep_wide_configure<TF, TV>(int, size_t); \
  template cudaError_t launch_sweep_wide<TF, TV>(const SweepArgs<TF, TV>&, int, int, size_t, cudaStream_t);
VTM_WIDE_INST(float, float)
VTM_WIDE_INST(double, double)
VTM_WIDE_INST(double, float)

}  // namespace vtm
