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
// s_off * 1024.  Inside a tile the layout is lane-major: element (row i, column c) sits at
// ((c / V) * 32 + i) * V + c % V with V = 16 / sizeof(T), so that one 16-byte load per lane gives
// every lane V consecutive entries of its own row.  Ports beyond n_ports are zero.
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
    S[t * kNB * kNB + ((col / V) * kNB + row) * V + col % V] =
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
// Shared memory: s (n_pad_ports x R) and the accumulator y (same size).
template <typename T, int R>
__global__ void __launch_bounds__(kSweepThreads, 2) k_port_sweep(const PortArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using VT = typename Vec16<T>::type;
  constexpr int V = Vec16<T>::V;
  constexpr int NL = kNB / V;  // 16-byte loads per lane per tile
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int np = pd.nports;
  if (np == 0) return;
  const int nt = (np + kNB - 1) / kNB;
  const int npad = nt * kNB;
  T* sv = reinterpret_cast<T*>(smem);
  T* yv = sv + (size_t)npad * R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // s_q = sum_e w_in[e] / Z_e, w_in[e] = w_prev[twin[e]]
  for (int i = tid; i < npad * R; i += kSweepThreads) {
    const int q = i / R, r = i % R;
    T acc = T(0);
    if (q < np) {
      const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
      for (int e = e0; e < e1; ++e) acc += a.wprev[(size_t)a.twin[e] * R + r] * a.invz[e];
    }
    sv[i] = acc;
    yv[i] = T(0);
  }
  __syncthreads();

  // y = S_j s over the stored lower block triangle: tile (I, J) adds T s_J to y_I and, off the
  // diagonal, T^T s_I to y_J
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  const VT* Sb = reinterpret_cast<const VT*>(a.S + pd.s_off * kNB * kNB);
  for (int t = warp; t < ntiles; t += kSweepThreads / 32) {
    int I, J;
    tile_of(t, I, J);
    const VT* tp = Sb + (int64_t)t * (kNB * kNB / V);
    VT v[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) v[k] = __ldg(tp + k * kNB + lane);
    const T* sJ = sv + (size_t)J * kNB * R;
    const T* sI = sv + (size_t)I * kNB * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // row part: lane = row of the tile
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NL; ++k)
#pragma unroll
        for (int c = 0; c < V; ++c) acc += Vec16<T>::get(v[k], c) * sJ[(k * V + c) * R + r];
      atomicAdd(&yv[((size_t)I * kNB + lane) * R + r], acc);
      if (I != J) {
        // column part: p[c] = T[lane][c] s_I[lane], summed over the lanes by a reduce-scatter
        // (after it, lane c holds column c)
        const T si = sI[lane * R + r];
        T p[kNB];
#pragma unroll
        for (int k = 0; k < NL; ++k)
#pragma unroll
          for (int c = 0; c < V; ++c) p[k * V + c] = Vec16<T>::get(v[k], c) * si;
#pragma unroll
        for (int h = kNB / 2; h >= 1; h >>= 1) {
          const bool upper = (lane & h) != 0;
#pragma unroll
          for (int i = 0; i < h; ++i) {
            const T send = upper ? p[i] : p[i + h];
            const T keep = upper ? p[i + h] : p[i];
            p[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
          }
        }
        atomicAdd(&yv[((size_t)J * kNB + lane) * R + r], p[0]);
      }
    }
  }
  __syncthreads();

  // w_out[e] = 2 (u_base + y)_q - w_in[e]
  for (int i = tid; i < np * R; i += kSweepThreads) {
    const int q = i / R, r = i % R;
    const T u = a.ubase[(size_t)(pd.port_off + q) * R + r] + yv[i];
    const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
    for (int e = e0; e < e1; ++e) a.wnext[(size_t)e * R + r] = T(2) * u - a.wprev[(size_t)a.twin[e] * R + r];
  }
}

size_t port_sweep_smem_bytes(size_t elem, int R, int max_ports) {
  const size_t npad = (size_t)((max_ports + kNB - 1) / kNB) * kNB;
  return 2 * npad * R * elem;
}

template <typename T>
cudaError_t port_sweep_configure(int R, size_t smem) {
  switch (R) {
    case 1: return cudaFuncSetAttribute(k_port_sweep<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 2: return cudaFuncSetAttribute(k_port_sweep<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 4: return cudaFuncSetAttribute(k_port_sweep<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 8: return cudaFuncSetAttribute(k_port_sweep<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_port_sweep(const PortArgs<T>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  switch (R) {
    case 1: k_port_sweep<T, 1><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 2: k_port_sweep<T, 2><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 4: k_port_sweep<T, 4><<<npieces, kSweepThreads, smem, st>>>(a); break;
    case 8: k_port_sweep<T, 8><<<npieces, kSweepThreads, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
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
  template cudaError_t port_sweep_configure<T>(int, size_t);                                                   \
  template cudaError_t launch_port_sweep<T>(const PortArgs<T>&, int, int, size_t, cudaStream_t);               \
  template cudaError_t launch_gather_port_response<T>(const PieceDesc*, int, const int32_t*, int, int, const T*, \
                                                      T*, cudaStream_t);                                        \
  template cudaError_t launch_gather_ports<T>(const PieceDesc*, int, const int32_t*, int, const T*, T*, cudaStream_t);
VTM_PORT_INST(float)
VTM_PORT_INST(double)

}  // namespace vtm
