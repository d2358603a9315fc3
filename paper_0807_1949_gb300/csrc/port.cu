// Port-response form of the VTM sweep.
//
// A sweep only needs each subgraph's port values u = P^T x_j, and x_j = K_j^{-1}(b̃_j + P s) with
// s_q = sum_{e at port q} w_in[e] / Z_e (eq. 5.8).  So u = u_base + S_j s with the port response
// S_j = P^T K_j^{-1} P (the open-circuit impedance matrix of Def. 7.1 taken over all ports at once,
// the Schur complement of the interior in K_j^{-1}, cf. eq. A3.3) and u_base = P^T K_j^{-1} b̃_j.
// The outgoing waves are w_out[e] = 2 u_q - w_in[e] (eq. 5.6), exactly as in the band sweep; only
// the way u is obtained differs.  S_j is symmetric, so only its lower block triangle is stored.
//
// Storage of S_j: 32 x 32 tiles (I, J), J <= I, in the order I (I + 1) / 2 + J, from element offset
// s_off * 1024.  Inside a tile lane L = 4 a + b of the warp owns the 4 x 8 patch of rows
// 4a .. 4a+3 and columns 8b .. 8b+7; patch entry p = (i mod 4) * 8 + (c mod 8) of element (i, c)
// sits at ((p / V) * 32 + L) * V + p mod V with V = 16 / sizeof(entry), so that the k-th 16-byte
// load of all lanes reads 512 contiguous bytes.  The row part T s_J then sums over 4 lanes and the
// column part T^T s_I over 8 lanes (short reduce-scatters).  Ports beyond n_ports are zero.
//
// FP16 storage (FP32 solvers): the same tiles as IEEE half, V = 8, each tile divided by its own
// largest entry (kept per tile in FP32); products and accumulation stay in FP32 and each tile's two
// reduced sums are scaled back before they enter y.  It halves the bytes of the sweep; its rounding
// (2^-11 of each tile's largest entry) is absorbed by the FP64 defect correction, and the solver
// returns to FP32 storage if a correction step stops gaining a digit.
#include <cuda_fp16.h>

#include "kernels.h"

namespace vtm {

namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int V = 4;
  __device__ static float get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int V = 2;
  __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
};

// Position of element (i, c) of a tile in the patch layout, V entries per 16 bytes.
__host__ __device__ __forceinline__ int patch_pos(int i, int c, int V) {
  const int L = (i / 4) * 4 + c / 8, p = (i % 4) * 8 + (c % 8);
  return ((p / V) * kNB + L) * V + p % V;
}

// The raw 16-byte vectors of this lane's patch (kNB entries of type TS), loaded ahead of use.
template <typename TS>
struct RawPatch {
  uint4 v[kNB * sizeof(TS) / 16];
};

template <typename TS>
__device__ __forceinline__ void load_raw(const TS* tile, int lane, RawPatch<TS>& r) {
  const uint4* tp = reinterpret_cast<const uint4*>(tile);
#pragma unroll
  for (int k = 0; k < (int)(kNB * sizeof(TS) / 16); ++k) r.v[k] = __ldg(tp + k * kNB + lane);
}

__device__ __forceinline__ void widen(const RawPatch<float>& r, float (&row)[kNB]) {
#pragma unroll
  for (int k = 0; k < kNB / 4; ++k) {
    row[4 * k] = __uint_as_float(r.v[k].x);
    row[4 * k + 1] = __uint_as_float(r.v[k].y);
    row[4 * k + 2] = __uint_as_float(r.v[k].z);
    row[4 * k + 3] = __uint_as_float(r.v[k].w);
  }
}

__device__ __forceinline__ void widen(const RawPatch<double>& r, double (&row)[kNB]) {
#pragma unroll
  for (int k = 0; k < kNB / 2; ++k) {
    row[2 * k] = __hiloint2double((int)r.v[k].y, (int)r.v[k].x);
    row[2 * k + 1] = __hiloint2double((int)r.v[k].w, (int)r.v[k].z);
  }
}

__device__ __forceinline__ void widen(const RawPatch<__half>& r, float (&row)[kNB]) {
#pragma unroll
  for (int k = 0; k < kNB / 8; ++k) {
    const uint32_t w[4] = {r.v[k].x, r.v[k].y, r.v[k].z, r.v[k].w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[j]));
      row[k * 8 + 2 * j] = f.x;
      row[k * 8 + 2 * j + 1] = f.y;
    }
  }
}

__device__ __forceinline__ void tile_of(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

}  // namespace

__host__ __device__ int64_t port_tiles(int nports) {
  const int64_t nt = (nports + kNB - 1) / kNB;
  return nt * (nt + 1) / 2;
}

// S_j columns from unit-source solves: column cc = b * Rs + r of S_j is x at the ports for the
// unit source at port cc (xc holds copies x Rs).  Only tiles with I >= J are written.
template <typename T>
__global__ void k_gather_port_response(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local,
                                       int Rs, int b, const T* __restrict__ xc, T* __restrict__ S) {
  const PieceDesc pd = pieces[blockIdx.x];
  constexpr int V = Vec16<T>::V;
  for (int i = threadIdx.x; i < pd.nports * Rs; i += blockDim.x) {
    const int q = i / Rs, r = i % Rs;
    const int cc = b * Rs + r;
    if (cc >= pd.nports) continue;
    const int I = q / kNB, J = cc / kNB;
    if (I < J) continue;
    const int row = q % kNB, col = cc % kNB;
    const int64_t t = pd.s_off + (int64_t)I * (I + 1) / 2 + J;
    S[t * kNB * kNB + patch_pos(row, col, V)] =
        xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * Rs + r];
  }
}

// u_base[port][r] = x_j at the port copy (xc from a sweep with zero incident waves).
template <typename T>
__global__ void k_gather_ports(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local, int R,
                               const T* __restrict__ xc, T* __restrict__ ubase) {
  const PieceDesc pd = pieces[blockIdx.x];
  for (int i = threadIdx.x; i < pd.nports * R; i += blockDim.x) {
    const int q = i / R, r = i % R;
    ubase[(size_t)(pd.port_off + q) * R + r] = xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * R + r];
  }
}

// One sweep in port-response form, one CTA per subgraph, R right-hand sides.
// Shared memory: s (n_pad_ports x R), the accumulator y (same size) and, with DET, one accumulator
// of the same size per warp.  Warp w takes the tiles w, w + 8, ... of the stored lower block
// triangle (so the eight warps stream neighbouring tiles).  With DET every warp adds its tiles'
// row and column parts to its own accumulator (in each add the 32 lanes hit 32 different ports),
// and the accumulators are summed in warp order at the end: identical runs agree bit for bit.
// Without DET (the accumulators would not fit) the warps add to y with shared-memory atomics.
template <typename T, typename TS, int R, bool DET>
__global__ void __launch_bounds__(kSweepThreads, sizeof(TS) == 2 ? 3 : 2) k_port_sweep(const PortArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int np = pd.nports;
  if (np == 0) return;
  const int nt = (np + kNB - 1) / kNB;
  const int npad = nt * kNB;
  T* sv = reinterpret_cast<T*>(smem);
  T* yv = sv + (size_t)npad * R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kSweepThreads / 32;
  T* const yacc = DET ? yv + (size_t)(1 + warp) * npad * R : yv;  // where this warp adds its parts
  if constexpr (DET) {
    for (int i = tid; i < kWarps * npad * R; i += kSweepThreads) yv[(size_t)npad * R + i] = T(0);
  }

  // s_q = sum_e w_in[e] / Z_e, w_in[e] = w_prev[twin[e]]; kU entries per thread at a time, their
  // end ranges, twins and waves loaded in three independent rounds
  constexpr int kU = 4;
  for (int i0 = tid; i0 < npad * R; i0 += kSweepThreads * kU) {
    int e0[kU], e1[kU], tw[kU];
    T iz[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = (i0 + u * kSweepThreads) / R;
      e0[u] = e1[u] = 0;
      if (q < np) {
        e0[u] = a.port_end_ptr[pd.port_off + q];
        e1[u] = a.port_end_ptr[pd.port_off + q + 1];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      tw[u] = (e1[u] > e0[u]) ? a.twin[e0[u]] : 0;
      iz[u] = (e1[u] > e0[u]) ? a.invz[e0[u]] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kSweepThreads;
      if (i >= npad * R) break;
      const int r = i % R;
      T acc = (e1[u] > e0[u]) ? a.wprev[(size_t)tw[u] * R + r] * iz[u] : T(0);
      for (int e = e0[u] + 1; e < e1[u]; ++e) acc += a.wprev[(size_t)a.twin[e] * R + r] * a.invz[e];
      if (a.cpl.ptr && i / R < np) acc += coupling_current<T, T>(a.cpl, pd.port_off + i / R, r, R, a.wprev);
      sv[i] = acc;
      yv[i] = T(0);
    }
  }
  __syncthreads();

  // y = S_j s over the stored lower block triangle: tile (I, J) adds T s_J to y_I and, off the
  // diagonal, T^T s_I to y_J.
  const TS* Sb;
  if constexpr (sizeof(TS) == 2) Sb = static_cast<const TS*>(a.Sh) + pd.s_off * kNB * kNB;
  else Sb = reinterpret_cast<const TS*>(a.S) + pd.s_off * kNB * kNB;
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  const int pa = lane >> 2, pb = lane & 3;  // patch: rows 4 pa .. +3, columns 8 pb .. +7
  // each warp keeps the next tile's loads in flight while it works on the current one
  RawPatch<TS> cur, nxt;
  // FP16 storage: each tile was divided by its own largest |entry|; the two reduced sums of a
  // tile are multiplied back before they are added to y
  const float* tsc = (sizeof(TS) == 2) ? a.scale + pd.s_off : nullptr;
  T sc_cur = T(1), sc_nxt = T(1);
  if (warp < ntiles) {
    load_raw(Sb + (int64_t)warp * kNB * kNB, lane, cur);
    if constexpr (sizeof(TS) == 2) sc_cur = (T)tsc[warp];
  }
  for (int t = warp; t < ntiles; t += kWarps) {
    if (t + kWarps < ntiles) {
      load_raw(Sb + (int64_t)(t + kWarps) * kNB * kNB, lane, nxt);
      if constexpr (sizeof(TS) == 2) sc_nxt = (T)tsc[t + kWarps];
    }
    int I, J;
    tile_of(t, I, J);
    T pt[kNB];
    widen(cur, pt);
    cur = nxt;
    const T sc = sc_cur;
    sc_cur = sc_nxt;
    const T* sJ = sv + ((size_t)J * kNB + 8 * pb) * R;
    const T* sI = sv + ((size_t)I * kNB + 4 * pa) * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // row part: 4 partial row sums over this lane's 8 columns, reduce-scattered over the 4 lanes
      // of the same row group (xor 2, 1): lane (pa, pb) ends with row 4 pa + pb
      T rp[4];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        T acc = T(0);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc += pt[ii * 8 + jj] * sJ[jj * R + r];
        rp[ii] = acc;
      }
#pragma unroll
      for (int h = 2; h >= 1; h >>= 1) {
        const bool upper = (pb & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
          const T send = upper ? rp[i] : rp[i + h];
          const T keep = upper ? rp[i + h] : rp[i];
          rp[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
      }
      {
        const T v = (sizeof(TS) == 2) ? rp[0] * sc : rp[0];
        T* at = &yacc[((size_t)I * kNB + 4 * pa + pb) * R + r];
        if constexpr (DET) *at += v;
        else atomicAdd(at, v);
      }
      if (I != J) {
        // column part: 8 partial column sums over this lane's 4 rows, reduce-scattered over the 8
        // lanes of the same column group (xor 16, 8, 4): lane (pa, pb) ends with column 8 pb + pa
        T cp[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          T acc = T(0);
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) acc += pt[ii * 8 + jj] * sI[ii * R + r];
          cp[jj] = acc;
        }
#pragma unroll
        for (int h = 4; h >= 1; h >>= 1) {
          const bool upper = (pa & h) != 0;
#pragma unroll
          for (int i = 0; i < h; ++i) {
            const T send = upper ? cp[i] : cp[i + h];
            const T keep = upper ? cp[i + h] : cp[i];
            cp[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4 * h);
          }
        }
        const T v = (sizeof(TS) == 2) ? cp[0] * sc : cp[0];
        T* at = &yacc[((size_t)J * kNB + 8 * pb + pa) * R + r];
        if constexpr (DET) *at += v;
        else atomicAdd(at, v);
      }
    }
  }
  __syncthreads();
  if constexpr (DET) {
    // y = the warps' accumulators, summed in warp order
    for (int i = tid; i < npad * R; i += kSweepThreads) {
      T v = T(0);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) v += yv[(size_t)(1 + w) * npad * R + i];
      yv[i] = v;
    }
    __syncthreads();
  }

  // w_out[e] = 2 (u_base + y)_q - w_in[e]
  for (int i0 = tid; i0 < np * R; i0 += kSweepThreads * kU) {
    int e0[kU], e1[kU], tw[kU];
    T ub[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kSweepThreads;
      e0[u] = e1[u] = 0;
      ub[u] = T(0);
      if (i < np * R) {
        const int q = i / R;
        e0[u] = a.port_end_ptr[pd.port_off + q];
        e1[u] = a.port_end_ptr[pd.port_off + q + 1];
        ub[u] = a.ubase[(size_t)pd.port_off * R + i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) tw[u] = (e1[u] > e0[u]) ? a.twin[e0[u]] : 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * kSweepThreads;
      if (i >= np * R) break;
      const int r = i % R;
      const T uu = ub[u] + yv[i];
      a.wnext[(size_t)e0[u] * R + r] = T(2) * uu - a.wprev[(size_t)tw[u] * R + r];
      for (int e = e0[u] + 1; e < e1[u]; ++e) a.wnext[(size_t)e * R + r] = T(2) * uu - a.wprev[(size_t)a.twin[e] * R + r];
    }
  }
}

size_t port_sweep_smem_bytes(size_t elem, int R, int max_ports, bool det) {
  const size_t npad = (size_t)((max_ports + kNB - 1) / kNB) * kNB;
  return (det ? 2 + kSweepThreads / 32 : 2) * npad * R * elem;
}

bool port_sweep_det_fits(size_t elem, int R, int max_ports) {
  return port_sweep_smem_bytes(elem, R, max_ports, true) <= kPortDetSmem;
}

template <typename T, typename TS, bool DET>
static cudaError_t port_configure_ts(int R, size_t smem) {
  const int b = (int)smem;
  switch (R) {
    case 1: return cudaFuncSetAttribute(k_port_sweep<T, TS, 1, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    case 2: return cudaFuncSetAttribute(k_port_sweep<T, TS, 2, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    case 4: return cudaFuncSetAttribute(k_port_sweep<T, TS, 4, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    case 8: return cudaFuncSetAttribute(k_port_sweep<T, TS, 8, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t port_sweep_configure(int R, size_t smem, bool det) {
  cudaError_t e = det ? port_configure_ts<T, T, true>(R, smem) : port_configure_ts<T, T, false>(R, smem);
  if constexpr (sizeof(T) == 4) {
    if (e == cudaSuccess) e = det ? port_configure_ts<T, __half, true>(R, smem) : port_configure_ts<T, __half, false>(R, smem);
  }
  return e;
}

template <typename T, typename TS, bool DET>
static cudaError_t port_launch_ts(const PortArgs<T>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  switch (R) {
    case 1: k_port_sweep<T, TS, 1, DET><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 2: k_port_sweep<T, TS, 2, DET><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 4: k_port_sweep<T, TS, 4, DET><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 8: k_port_sweep<T, TS, 8, DET><<<npieces, kSweepThreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_port_sweep(const PortArgs<T>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (a.Sh) return a.det ? port_launch_ts<T, __half, true>(a, R, npieces, smem, st)
                           : port_launch_ts<T, __half, false>(a, R, npieces, smem, st);
  }
  return a.det ? port_launch_ts<T, T, true>(a, R, npieces, smem, st) : port_launch_ts<T, T, false>(a, R, npieces, smem, st);
}

// FP16 copy of the FP32 tiles of one subgraph per CTA, one warp per tile: each tile is divided by
// its largest |entry| (1 if all zero), kept per tile in scale[s_off + t], and re-laid out from the
// float patch layout ((p/4)*32 + L)*4 + p%4 to the half patch layout ((p/8)*32 + L)*8 + p%8.  A scale
// per tile keeps the small far-field blocks of S_j at full FP16 precision.
__global__ void k_port_to_half(const PieceDesc* __restrict__ pieces, const float* __restrict__ S,
                               __half* __restrict__ Sh, float* __restrict__ scale) {
  const PieceDesc pd = pieces[blockIdx.x];
  const int64_t nt = port_tiles(pd.nports);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t t = warp; t < nt; t += blockDim.x >> 5) {
    const float* src = S + (pd.s_off + t) * kNB * kNB;
    __half* dst = Sh + (pd.s_off + t) * kNB * kNB;
    float m = 0.f;
    for (int k = lane; k < kNB * kNB; k += 32) m = fmaxf(m, fabsf(src[k]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float sc = m > 0.f ? m : 1.f;
    if (lane == 0) scale[pd.s_off + t] = sc;
    const float inv = 1.f / sc;
    for (int k = lane; k < kNB * kNB; k += 32) {
      const int L = (k / 4) % kNB, p = (k / 128) * 4 + (k % 4);
      dst[((p / 8) * kNB + L) * 8 + (p % 8)] = __float2half_rn(src[k] * inv);
    }
  }
}

cudaError_t launch_port_to_half(const PieceDesc* pieces, int npieces, const float* S, __half* Sh, float* scale,
                                cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_port_to_half<<<npieces, kSweepThreads, 0, st>>>(pieces, S, Sh, scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_port_response(const PieceDesc* pieces, int npieces, const int32_t* port_local, int Rs, int b,
                                        const T* xc, T* S, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_gather_port_response<T><<<npieces, 256, 0, st>>>(pieces, port_local, Rs, b, xc, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_ports(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, const T* xc,
                                T* ubase, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_gather_ports<T><<<npieces, 256, 0, st>>>(pieces, port_local, R, xc, ubase);
  return cudaGetLastError();
}

#define VTM_PORT_INST(T)                                                                                       \
  template cudaError_t port_sweep_configure<T>(int, size_t, bool);                                             \
  template cudaError_t launch_port_sweep<T>(const PortArgs<T>&, int, int, size_t, cudaStream_t);               \
  template cudaError_t launch_gather_port_response<T>(const PieceDesc*, int, const int32_t*, int, int, const T*, \
                                                      T*, cudaStream_t);                                        \
  template cudaError_t launch_gather_ports<T>(const PieceDesc*, int, const int32_t*, int, const T*, T*, cudaStream_t);
VTM_PORT_INST(float)
VTM_PORT_INST(double)

}  // namespace vtm
