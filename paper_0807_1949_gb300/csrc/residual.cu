// Vector kernels around the sweeps: source splitting (§4 step 3), assembly of the solution from the
// copies (mean of the copies; at the fixed point all copies agree, Thm 4.1), and the FP64 residual
// b - A x with per-right-hand-side squared norms (the convergence test of Table 1 step 6).
#include <type_traits>

#include "kernels.h"

namespace vtm {

namespace {
constexpr int kMaxR = kMaxRhs;
constexpr int kBS = 256;
constexpr int kNormRows = 8;  // rows per thread in the fixed-order norm kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of R values per thread, accumulated into norms[r] with one atomic per block.
__device__ void block_accumulate(const double* v, int R, double* norms) {
  __shared__ double red[kBS / 32][kMaxR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) {
    if (r >= R) break;
    const double s = warp_sum(v[r]);
    if (lane == 0) red[warp][r] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int r = 0; r < kMaxR; ++r) {
      if (r >= R) break;
      double s = lane < kBS / 32 ? red[lane][r] : 0.0;
      s = warp_sum(s);
      if (lane == 0) atomicAdd(&norms[r], s);
    }
  }
}
}  // namespace

// Thread (copy c, columns 4 g .. 4 g + 3): the four values of a copy go out in one vector store
// (b̃ is copies x R with R contiguous; R % 4 == 0 here, other R one column per thread).
template <typename T, int CG>
__global__ void k_split(int64_t ncopies, int R, const int64_t* __restrict__ copy_vertex, const double* __restrict__ share,
                        const double* __restrict__ src, int64_t ld, T* __restrict__ bt) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * CG;
  if (c >= ncopies) return;
  const int64_t v = copy_vertex[c];
  const double s = share[c];
  T o[CG];
#pragma unroll
  for (int j = 0; j < CG; ++j) o[j] = (T)(s * src[v + (int64_t)(r0 + j) * ld]);
  T* q = bt + c * R + r0;
  if constexpr (CG == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
  } else if constexpr (CG == 4 && sizeof(T) == 8) {
    reinterpret_cast<double2*>(q)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2*>(q)[1] = make_double2(o[2], o[3]);
  } else {
#pragma unroll
    for (int j = 0; j < CG; ++j) q[j] = o[j];
  }
}

// Thread (vertex or row i, column group blockIdx.y): RG right-hand sides per thread, so that the
// row of A (or the copy list of the vertex) is read once per group and each column's accesses to
// the column-major vectors are coalesced across neighbouring threads.
template <typename T, int RG>
__global__ void k_assemble(int64_t n, int R, const int64_t* __restrict__ vc_ptr, const int64_t* __restrict__ vc_copy,
                           const T* __restrict__ xc, const double* __restrict__ xbase, double* __restrict__ xt, int64_t ld) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * RG;
  if (i >= n) return;
  const int64_t lo = vc_ptr[i], hi = vc_ptr[i + 1];
  // FP32 copies: their mean in FP32 (the copies carry FP32 rounding already), one FP64 add
  using A = typename std::conditional<sizeof(T) == 4, float, double>::type;
  const A inv = A(1) / (A)(hi - lo);
  A s[RG];
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) s[rr] = A(0);
  for (int64_t k = lo; k < hi; ++k) {
    const T* p = xc + vc_copy[k] * R + r0;  // the copy's RG values are contiguous (and 16-byte
                                            // aligned when RG is 4 or 8: R and r0 are multiples of RG)
    if constexpr (RG % 4 == 0 && sizeof(T) == 4) {
#pragma unroll
      for (int g = 0; g < RG / 4; ++g) {
        const float4 v = reinterpret_cast<const float4*>(p)[g];
        s[4 * g] += v.x, s[4 * g + 1] += v.y, s[4 * g + 2] += v.z, s[4 * g + 3] += v.w;
      }
    } else if constexpr (RG % 2 == 0 && sizeof(T) == 8) {
#pragma unroll
      for (int g = 0; g < RG / 2; ++g) {
        const double2 v = reinterpret_cast<const double2*>(p)[g];
        s[2 * g] += v.x, s[2 * g + 1] += v.y;
      }
    } else {
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) s[rr] += (A)p[rr];
    }
  }
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) {
    const int64_t at = i + (int64_t)(r0 + rr) * ld;
    xt[at] = (xbase ? xbase[at] : 0.0) + (double)(s[rr] * inv);
  }
}

template <int RG>
__global__ void k_residual(int64_t n, int R, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ b, int64_t ldb,
                           const double* __restrict__ x, int64_t ldx, double* __restrict__ res, int64_t ldr,
                           double* norms) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r0 = blockIdx.y * RG;
  double sq[kMaxR];
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) sq[r] = 0.0;
  if (i < n) {
    const int64_t lo = rowptr[i], hi = rowptr[i + 1];
    double ax[RG];
#pragma unroll
    for (int rr = 0; rr < RG; ++rr) ax[rr] = 0.0;
    for (int64_t k = lo; k < hi; ++k) {
      const double v = val[k];
      const double* xk = x + col[k];
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) ax[rr] += v * xk[(int64_t)(r0 + rr) * ldx];
    }
#pragma unroll
    for (int rr = 0; rr < RG; ++rr) {
      const double ri = b[i + (int64_t)(r0 + rr) * ldb] - ax[rr];
      if (res) res[i + (int64_t)(r0 + rr) * ldr] = ri;
      sq[rr] = ri * ri;
    }
  }
  block_accumulate(sq, RG, norms + r0);
}

// The same residual with fixed-order sums: block (x, y) writes the squared norms of its rows'
// residuals, column by column, to part[r * gridDim.x + x] (each thread sums kNormRows rows, then the
// block's warps are summed in warp order), and k_finish_norms adds each column's partials in index
// order.  The row's entries of A are loaded eight at a time before the products, so that the loads
// of x for all of them are in flight together.  FP64 arithmetic is the bound on this GPU (a small
// fraction of the FP32 rate), so every thread covers several rows before the butterfly sums.
template <int RG>
__global__ void __launch_bounds__(kBS) k_residual_part(int64_t n, int R, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col, const double* __restrict__ val,
                                                        const double* __restrict__ b, int64_t ldb,
                                                        const double* __restrict__ x, int64_t ldx,
                                                        double* __restrict__ res, int64_t ldr, double* __restrict__ part) {
  const int r0 = blockIdx.y * RG;
  double sq[RG];
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) sq[rr] = 0.0;
  for (int j = 0; j < kNormRows; ++j) {
    const int64_t i = (blockIdx.x * (int64_t)kNormRows + j) * blockDim.x + threadIdx.x;
    if (i < n) {
      const int64_t lo = rowptr[i], hi = rowptr[i + 1];
      double ax[RG];
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) ax[rr] = 0.0;
      for (int64_t k0 = lo; k0 < hi; k0 += 8) {
        int c[8];
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          c[u] = k0 + u < hi ? col[k0 + u] : 0;
          v[u] = k0 + u < hi ? val[k0 + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (k0 + u < hi) {
            const double* xk = x + c[u] + (int64_t)r0 * ldx;
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) ax[rr] += v[u] * xk[(int64_t)rr * ldx];
          }
        }
      }
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) {
        const double ri = b[i + (int64_t)(r0 + rr) * ldb] - ax[rr];
        if (res) res[i + (int64_t)(r0 + rr) * ldr] = ri;
        sq[rr] = fma(ri, ri, sq[rr]);
      }
    }
  }
  __shared__ double red[kBS / 32][RG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) {
    const double t = warp_sum(sq[rr]);
    if (lane == 0) red[warp][rr] = t;
  }
  __syncthreads();
  if (threadIdx.x < RG) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kBS / 32; ++w) t += red[w][threadIdx.x];
    part[(int64_t)(r0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

template <int RG>
__global__ void __launch_bounds__(kBS) k_sqnorm_part(int64_t n, const double* __restrict__ v, int64_t ld,
                                                      double* __restrict__ part) {
  const int r0 = blockIdx.y * RG;
  __shared__ double red[kBS / 32][RG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double sq[RG];
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) sq[rr] = 0.0;
  for (int j = 0; j < kNormRows; ++j) {
    const int64_t i = (blockIdx.x * (int64_t)kNormRows + j) * blockDim.x + threadIdx.x;
#pragma unroll
    for (int rr = 0; rr < RG; ++rr) {
      const double t = i < n ? v[i + (int64_t)(r0 + rr) * ld] : 0.0;
      sq[rr] = fma(t, t, sq[rr]);
    }
  }
#pragma unroll
  for (int rr = 0; rr < RG; ++rr) {
    const double w = warp_sum(sq[rr]);
    if (lane == 0) red[warp][rr] = w;
  }
  __syncthreads();
  if (threadIdx.x < RG) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kBS / 32; ++w) t += red[w][threadIdx.x];
    part[(int64_t)(r0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

// norms[r] = sum of part[r * nparts + 0 .. nparts - 1]: thread t adds the partials t, t + kBS, ... in
// order, then the block's sums are combined in a fixed tree.
__global__ void __launch_bounds__(kBS) k_finish_norms(int nparts, const double* __restrict__ part, double* norms) {
  const int r = blockIdx.x;
  const double* p = part + (int64_t)r * nparts;
  double t = 0.0;
  for (int j = threadIdx.x; j < nparts; j += kBS) t += p[j];
  __shared__ double red[kBS / 32];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < kBS / 32 ? red[threadIdx.x] : 0.0;
    u = warp_sum(u);
    if (threadIdx.x == 0) norms[r] = u;
  }
}

__global__ void k_sqnorm(int64_t n, int R, const double* __restrict__ v, int64_t ld, double* norms) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double sq[kMaxR];
#pragma unroll
  for (int r = 0; r < kMaxR; ++r) sq[r] = 0.0;
  if (i < n)
#pragma unroll
    for (int r = 0; r < kMaxR; ++r) {
      if (r >= R) break;
      const double t = v[i + r * ld];
      sq[r] = t * t;
    }
  block_accumulate(sq, R, norms);
}

__global__ void k_copy2d(int64_t n, int R, const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int r = 0; r < R; ++r) dst[i + r * ldd] = src[i + r * lds];
}

template <typename T>
__global__ void k_unit_rhs(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local, int R, int b,
                           T* __restrict__ bt) {
  const PieceDesc pd = pieces[blockIdx.x];
  T* p = bt + (size_t)pd.copy_off * R;
  for (int i = threadIdx.x; i < pd.n * R; i += blockDim.x) p[i] = T(0);
  __syncthreads();
  const int r = threadIdx.x;
  if (r < R) {
    const int q = b * R + r;
    if (q < pd.nports) p[(size_t)port_local[pd.port_off + q] * R + r] = T(1);
  }
}

template <typename T>
__global__ void k_gather_diag(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local, int R,
                              int b, const T* __restrict__ xc, double* __restrict__ g) {
  const PieceDesc pd = pieces[blockIdx.x];
  const int r = threadIdx.x;
  if (r < R) {
    const int q = b * R + r;
    if (q < pd.nports) g[pd.port_off + q] = (double)xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * R + r];
  }
}

static unsigned nblocks(int64_t n) { return (unsigned)((n + kBS - 1) / kBS); }
static unsigned nblocks_norm(int64_t n) { return (unsigned)((n + kBS * kNormRows - 1) / (kBS * kNormRows)); }

template <typename T>
cudaError_t launch_split(int64_t ncopies, int R, const int64_t* copy_vertex, const double* share, const double* src,
                         int64_t ld, T* bt, cudaStream_t st) {
  if (ncopies <= 0) return cudaSuccess;
  if (R % 4 == 0) k_split<T, 4><<<dim3(nblocks(ncopies), R / 4), kBS, 0, st>>>(ncopies, R, copy_vertex, share, src, ld, bt);
  else k_split<T, 1><<<dim3(nblocks(ncopies), R), kBS, 0, st>>>(ncopies, R, copy_vertex, share, src, ld, bt);
  return cudaGetLastError();
}

// Column groups of min(R, 8) right-hand sides (R is 1, 2, 4, 8, 16 or 32; other counts go one by one).
template <typename T>
cudaError_t launch_assemble(int64_t n, int R, const int64_t* vc_ptr, const int64_t* vc_copy, const T* xc,
                            const double* xbase, double* xt, int64_t ld, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned bx = nblocks(n);
  if (R % 8 == 0) k_assemble<T, 8><<<dim3(bx, R / 8), kBS, 0, st>>>(n, R, vc_ptr, vc_copy, xc, xbase, xt, ld);
  else if (R % 4 == 0) k_assemble<T, 4><<<dim3(bx, R / 4), kBS, 0, st>>>(n, R, vc_ptr, vc_copy, xc, xbase, xt, ld);
  else if (R % 2 == 0) k_assemble<T, 2><<<dim3(bx, R / 2), kBS, 0, st>>>(n, R, vc_ptr, vc_copy, xc, xbase, xt, ld);
  else k_assemble<T, 1><<<dim3(bx, R), kBS, 0, st>>>(n, R, vc_ptr, vc_copy, xc, xbase, xt, ld);
  return cudaGetLastError();
}

cudaError_t launch_residual(int64_t n, int R, const int64_t* rowptr, const int32_t* col, const double* val,
                            const double* b, int64_t ldb, const double* x, int64_t ldx, double* res, int64_t ldr,
                            double* norms, cudaStream_t st) {
  if (R > kMaxR || R < 1) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  const unsigned bx = nblocks(n);
  if (R % 8 == 0) k_residual<8><<<dim3(bx, R / 8), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, norms);
  else if (R % 4 == 0) k_residual<4><<<dim3(bx, R / 4), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, norms);
  else if (R % 2 == 0) k_residual<2><<<dim3(bx, R / 2), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, norms);
  else k_residual<1><<<dim3(bx, R), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, norms);
  return cudaGetLastError();
}

int64_t norm_parts(int64_t n) { return (int64_t)nblocks_norm(n); }

cudaError_t launch_residual_det(int64_t n, int R, const int64_t* rowptr, const int32_t* col, const double* val,
                                const double* b, int64_t ldb, const double* x, int64_t ldx, double* res, int64_t ldr,
                                double* part, double* norms, cudaStream_t st) {
  if (R > kMaxR || R < 1) return cudaErrorInvalidValue;
  if (n <= 0) return cudaMemsetAsync(norms, 0, R * sizeof(double), st);
  const unsigned bx = nblocks_norm(n);
  if (R % 8 == 0) k_residual_part<8><<<dim3(bx, R / 8), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, part);
  else if (R % 4 == 0) k_residual_part<4><<<dim3(bx, R / 4), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, part);
  else if (R % 2 == 0) k_residual_part<2><<<dim3(bx, R / 2), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, part);
  else k_residual_part<1><<<dim3(bx, R), kBS, 0, st>>>(n, R, rowptr, col, val, b, ldb, x, ldx, res, ldr, part);
  k_finish_norms<<<R, kBS, 0, st>>>((int)bx, part, norms);
  return cudaGetLastError();
}

cudaError_t launch_sqnorm_det(int64_t n, int R, const double* v, int64_t ld, double* part, double* norms,
                              cudaStream_t st) {
  if (R > kMaxR || R < 1) return cudaErrorInvalidValue;
  if (n <= 0) return cudaMemsetAsync(norms, 0, R * sizeof(double), st);
  const unsigned bx = nblocks_norm(n);
  if (R % 8 == 0) k_sqnorm_part<8><<<dim3(bx, R / 8), kBS, 0, st>>>(n, v, ld, part);
  else if (R % 4 == 0) k_sqnorm_part<4><<<dim3(bx, R / 4), kBS, 0, st>>>(n, v, ld, part);
  else if (R % 2 == 0) k_sqnorm_part<2><<<dim3(bx, R / 2), kBS, 0, st>>>(n, v, ld, part);
  else k_sqnorm_part<1><<<dim3(bx, R), kBS, 0, st>>>(n, v, ld, part);
  k_finish_norms<<<R, kBS, 0, st>>>((int)bx, part, norms);
  return cudaGetLastError();
}

cudaError_t launch_sqnorm(int64_t n, int R, const double* v, int64_t ld, double* norms, cudaStream_t st) {
  if (R > kMaxR) return cudaErrorInvalidValue;
  k_sqnorm<<<nblocks(n), kBS, 0, st>>>(n, R, v, ld, norms);
  return cudaGetLastError();
}

cudaError_t launch_copy2d(int64_t n, int R, const double* src, int64_t lds, double* dst, int64_t ldd, cudaStream_t st) {
  k_copy2d<<<nblocks(n), kBS, 0, st>>>(n, R, src, lds, dst, ldd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unit_rhs(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, int b, T* bt,
                            cudaStream_t st) {
  k_unit_rhs<T><<<npieces, 256, 0, st>>>(pieces, port_local, R, b, bt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_diag(const PieceDesc* pieces, int npieces, const int32_t* port_local, int R, int b,
                               const T* xc, double* g, cudaStream_t st) {
  k_gather_diag<T><<<npieces, 32, 0, st>>>(pieces, port_local, R, b, xc, g);
  return cudaGetLastError();
}

template cudaError_t launch_unit_rhs<float>(const PieceDesc*, int, const int32_t*, int, int, float*, cudaStream_t);
template cudaError_t launch_unit_rhs<double>(const PieceDesc*, int, const int32_t*, int, int, double*, cudaStream_t);
template cudaError_t launch_gather_diag<float>(const PieceDesc*, int, const int32_t*, int, int, const float*, double*,
                                               cudaStream_t);
template cudaError_t launch_gather_diag<double>(const PieceDesc*, int, const int32_t*, int, int, const double*,
                                                double*, cudaStream_t);
template cudaError_t launch_split<float>(int64_t, int, const int64_t*, const double*, const double*, int64_t, float*,
                                         cudaStream_t);
template cudaError_t launch_split<double>(int64_t, int, const int64_t*, const double*, const double*, int64_t, double*,
                                          cudaStream_t);
template cudaError_t launch_assemble<float>(int64_t, int, const int64_t*, const int64_t*, const float*, const double*,
                                            double*, int64_t, cudaStream_t);
template cudaError_t launch_assemble<double>(int64_t, int, const int64_t*, const int64_t*, const double*,
                                             const double*, double*, int64_t, cudaStream_t);

}  // namespace vtm
