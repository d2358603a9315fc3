// Local matrices of eq. 5.8 and their banded Cholesky factors, computed once per setup (§8: "the
// Cholesky factorization for one time, and the forward and backward substitution for the rest").
//
// K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T is assembled into the right-aligned band storage described
// in device.cuh, then factored in place by a blocked right-looking band Cholesky (kNB columns per
// step: factor the diagonal block with one warp in shared memory, solve the panel below it, update the
// trailing band).  Every diagonal block is finally replaced by the inverse of its triangular
// factor so that the substitution needs no sequential triangular solves.
#include "kernels.h"

namespace vtm {

template <typename T>
__global__ void k_build_band(int64_t ncopies, const int32_t* __restrict__ copy_piece, const PieceDesc* __restrict__ pieces,
                             const int64_t* __restrict__ l_rowptr, const int32_t* __restrict__ l_col,
                             const double* __restrict__ l_val, const int32_t* __restrict__ port_of_copy,
                             const int32_t* __restrict__ port_end_ptr, const double* __restrict__ invz, T* band,
                             int* status) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncopies) return;
  if (copy_piece[c] < 0) return;  // subgraph not part of this band
  const PieceDesc pd = pieces[copy_piece[c]];
  const int64_t l = c - pd.copy_off;
  const int off = pd.Wp - 1;
  T* row = band + pd.factor_off + l * pd.Wp;
  double extra = 0.0;
  const int q = port_of_copy[c];
  if (q >= 0)
    for (int e = port_end_ptr[q]; e < port_end_ptr[q + 1]; ++e) extra += invz[e];
  for (int64_t k = l_rowptr[c]; k < l_rowptr[c + 1]; ++k) {
    const int64_t col = l_col[k];
    if (col > l) continue;
    const int64_t d = l - col;
    if (d > off) {
      atomicExch(status, 1);
      continue;
    }
    double v = l_val[k];
    if (d == 0) v += extra;
    row[off - d] = (T)v;
  }
}

template <typename T>
__global__ void k_pad_rows(const PieceDesc* __restrict__ pieces, int npieces, int max_pad, T* band) {
  const int j = blockIdx.x;
  const PieceDesc pd = pieces[j];
  for (int r = pd.n + threadIdx.x; r < pd.n_pad; r += blockDim.x)
    band[pd.factor_off + (int64_t)r * pd.Wp + pd.Wp - 1] = T(1);
}

// One CTA (256 threads) per subgraph.  Shared memory: D (kNB x 33) and the panel P (w x 33).
template <typename T>
__global__ void __launch_bounds__(256) k_factor(const PieceDesc* __restrict__ pieces, T* band, int* status,
                                                int* piece_flag, T* diag0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* D = reinterpret_cast<T*>(smem_raw);
  T* P = D + kNB * 33;
  __shared__ int bad;   // 1: non-positive pivot, 2: pivot^2 < kFlagRatio * original diagonal
  const PieceDesc pd = pieces[blockIdx.x];
  T* B = band + pd.factor_off;
  const int Wp = pd.Wp, off = Wp - 1, w = pd.w, n_pad = pd.n_pad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) bad = 0;
  // original diagonal of K_j (rows are updated in place by earlier blocks)
  if (diag0)
    for (int r = tid; r < n_pad; r += blockDim.x) diag0[pd.row_off + r] = B[(int64_t)r * Wp + off];
  __syncthreads();
  for (int k0 = 0; k0 < n_pad; k0 += kNB) {
    // (a) diagonal block of the updated band
    for (int idx = tid; idx < kNB * kNB; idx += blockDim.x) {
      const int r = idx / kNB, c = idx % kNB;
      D[r * 33 + c] = (c <= r) ? B[(int64_t)(k0 + r) * Wp + off - (r - c)] : T(0);
    }
    __syncthreads();
    if (warp == 0) {
      // right-looking Cholesky of the block in shared memory, lane i owning row i: at step j lane j
      // takes the pivot, the lanes below scale their entry of column j and update their row
      const T d0 = diag0 ? diag0[pd.row_off + k0 + lane] : D[lane * 33 + lane];
      for (int j = 0; j < kNB; ++j) {
        if (lane == j) {
          T djj = D[j * 33 + j];
          if (!(djj > T(0))) {
            bad = 1;
            djj = T(1);
          } else if (djj < T(kFlagRatio) * d0 && bad == 0) {
            bad = 2;
          }
          D[j * 33 + j] = sqrt(djj);
        }
        __syncwarp();
        if (lane > j) D[lane * 33 + j] /= D[j * 33 + j];
        __syncwarp();
        if (lane > j) {
          const T lij = D[lane * 33 + j];
          for (int c = j + 1; c <= lane; ++c) D[lane * 33 + c] -= lij * D[c * 33 + j];
        }
        __syncwarp();
      }
      for (int c = lane + 1; c < kNB; ++c) D[lane * 33 + c] = T(0);
    }
    __syncthreads();
    // (b) panel: rows below the block within the band, L_IK = A_IK L_KK^{-T}
    int nrows = n_pad - k0 - kNB;
    if (nrows > w) nrows = w;
    if (nrows < 0) nrows = 0;
    for (int ri = tid; ri < nrows; ri += blockDim.x) {
      const int64_t i = k0 + kNB + ri;
      T x[kNB];
#pragma unroll
      for (int c = 0; c < kNB; ++c) {
        const int dist = (int)(i - (k0 + c));
        x[c] = (dist <= off) ? B[i * Wp + off - dist] : T(0);
      }
#pragma unroll
      for (int c = 0; c < kNB; ++c) {
        T s = x[c];
#pragma unroll
        for (int k = 0; k < c; ++k) s -= x[k] * D[c * 33 + k];
        x[c] = s / D[c * 33 + c];
      }
#pragma unroll
      for (int c = 0; c < kNB; ++c) {
        const int dist = (int)(i - (k0 + c));
        P[ri * 33 + c] = x[c];
        if (dist <= off) B[i * Wp + off - dist] = x[c];
      }
    }
    __syncthreads();
    // (c) trailing band update A_IJ -= L_IK L_JK^T (lower triangle of the w x w window)
    for (int ri = warp; ri < nrows; ri += blockDim.x / 32) {
      const T* pi = P + ri * 33;
      const int64_t i = k0 + kNB + ri;
      for (int cj = lane; cj <= ri; cj += 32) {
        const T* pj = P + cj * 33;
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < kNB; ++c) acc += pi[c] * pj[c];
        B[i * Wp + off - (ri - cj)] -= acc;
      }
    }
    // (d) replace the diagonal block by inv(L_KK) (column j by thread j)
    if (tid < kNB) {
      const int j = tid;
      T X[kNB];
#pragma unroll
      for (int i = 0; i < kNB; ++i) {
        if (i < j) {
          X[i] = T(0);
        } else if (i == j) {
          X[i] = T(1) / D[i * 33 + i];
        } else {
          T s = T(0);
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
  if (tid == 0 && bad) {
    if (piece_flag) piece_flag[blockIdx.x] = bad;
    else if (bad == 1) atomicExch(status, kStatusNotSpd);
  }
}

// U = L^T in the same band geometry, LEFT-aligned: entry d of row i holds U[i][i+d] = L[i+d][i]
// (d = 0 is the diagonal).  The diagonal blocks carry the transposed inverses, inv(L_KK)^T =
// inv(L_KK^T), so the back substitution runs in dot form on contiguous rows of U.
template <typename T>
__global__ void k_transpose_band(const PieceDesc* __restrict__ pieces, const T* __restrict__ L, T* __restrict__ U) {
  const PieceDesc pd = pieces[blockIdx.y];
  const int Wp = pd.Wp, off = Wp - 1;
  const int64_t total = (int64_t)pd.n_pad * Wp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / Wp;
    const int d = (int)(idx % Wp);
    T v = T(0);
    if (i + d < pd.n_pad) v = L[pd.factor_off + (i + d) * Wp + off - d];
    U[pd.factor_off + idx] = v;
  }
}

template <typename T>
cudaError_t launch_transpose_band(const PieceDesc* pieces, int npieces, const T* L, T* U, cudaStream_t st) {
  dim3 grid(64, npieces);
  k_transpose_band<T><<<grid, 256, 0, st>>>(pieces, L, U);
  return cudaGetLastError();
}

template cudaError_t launch_transpose_band<float>(const PieceDesc*, int, const float*, float*, cudaStream_t);
template cudaError_t launch_transpose_band<double>(const PieceDesc*, int, const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_build_band(int64_t ncopies, const int32_t* copy_piece, const PieceDesc* pieces,
                              const int64_t* l_rowptr, const int32_t* l_col, const double* l_val,
                              const int32_t* port_of_copy, const int32_t* port_end_ptr, const double* invz,
                              int npieces, int max_pad_rows, T* band, int* status, cudaStream_t st) {
  const int bs = 256;
  if (ncopies > 0)
    k_build_band<T><<<(unsigned)((ncopies + bs - 1) / bs), bs, 0, st>>>(ncopies, copy_piece, pieces, l_rowptr, l_col,
                                                                        l_val, port_of_copy, port_end_ptr, invz, band,
                                                                        status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pad_rows<T><<<npieces, 64, 0, st>>>(pieces, npieces, max_pad_rows, band);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_factor(const PieceDesc* pieces, int npieces, int max_w, T* band, int* status, int* piece_flag,
                          T* diag0, cudaStream_t st) {
  const size_t smem = sizeof(T) * 33 * (size_t)(kNB + (max_w > kNB ? max_w : kNB));
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor<T><<<npieces, 256, smem, st>>>(pieces, band, status, piece_flag, diag0);
  return cudaGetLastError();
}

template cudaError_t launch_build_band<float>(int64_t, const int32_t*, const PieceDesc*, const int64_t*, const int32_t*,
                                              const double*, const int32_t*, const int32_t*, const double*, int, int,
                                              float*, int*, cudaStream_t);
template cudaError_t launch_build_band<double>(int64_t, const int32_t*, const PieceDesc*, const int64_t*, const int32_t*,
                                               const double*, const int32_t*, const int32_t*, const double*, int, int,
                                               double*, int*, cudaStream_t);
template cudaError_t launch_factor<float>(const PieceDesc*, int, int, float*, int*, int*, float*, cudaStream_t);
template cudaError_t launch_factor<double>(const PieceDesc*, int, int, double*, int*, int*, double*, cudaStream_t);

}  // namespace vtm
