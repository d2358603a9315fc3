// Coupled virtual transmission lines (§7.2, Thm 7.1): the coupling current of every port.
//
// A bundle (the lines joining the same two subgraphs) may carry conductances y between pairs of
// its lines, so that its admittance is Y = diag(1/Z_t) + sum_p y_p (e_t - e_t')(e_t - e_t')^T.
// The diagonal part is the uncoupled method, applied by the sweep kernels themselves (the sum of
// w_in[e] / Z_e at each port); the coupled part adds, at the port of end e of line t,
//     sum over the pairs (t, t') of y (w_in[e] - w_in[e']),
// e' the end of t' at the same subgraph.  This kernel forms that sum for every port before the
// sweep; the pairs are stored per port (CSR) with the wave indices of their two incoming waves.
// Bytes: one pass over the pair list and two gathered waves per entry, ~1/20 of a port sweep.
#include "kernels.h"

namespace vtm {

template <typename T>
__global__ void k_couple(int nports, int R, const int32_t* __restrict__ cp_ptr, const int32_t* __restrict__ own,
                         const int32_t* __restrict__ oth, const T* __restrict__ y, const T* __restrict__ w,
                         T* __restrict__ cq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nports * R) return;
  const int q = (int)(i / R), r = (int)(i % R);
  T acc = T(0);
  for (int k = cp_ptr[q]; k < cp_ptr[q + 1]; ++k)
    acc += y[k] * (w[(size_t)own[k] * R + r] - w[(size_t)oth[k] * R + r]);
  cq[i] = acc;
}

template <typename T>
cudaError_t launch_couple(int nports, int R, const int32_t* cp_ptr, const int32_t* own, const int32_t* oth,
                          const T* y, const T* w, T* cq, cudaStream_t st) {
  const int64_t n = (int64_t)nports * R;
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  k_couple<T><<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(nports, R, cp_ptr, own, oth, y, w, cq);
  return cudaGetLastError();
}

template cudaError_t launch_couple<float>(int, int, const int32_t*, const int32_t*, const int32_t*, const float*,
                                          const float*, float*, cudaStream_t);
template cudaError_t launch_couple<double>(int, int, const int32_t*, const int32_t*, const int32_t*, const double*,
                                           const double*, double*, cudaStream_t);

}  // namespace vtm
