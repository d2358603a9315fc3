// Learned line impedance: a 3-layer perceptron 8 -> 64 -> 64 -> 1 (ReLU) that maps 8 local
// features of a line end to log Z (impedance matching, §7.1, governs convergence; the network
// replaces the input-impedance rule with impedances found by search).  Weights are held in BF16
// for the forward and backward passes (FP32 accumulation); Adam keeps an FP32 master copy.
//
// Parameter layout (P = 4801 floats): W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
// Forward / backward: one thread per sample; a CTA keeps the BF16 weights (as FP32 values) in
// shared memory.  The backward pass stores each tile's hidden activations and output gradients in
// shared memory and forms the weight gradients as tile GEMMs (sum over the tile's samples), with
// one atomic add per parameter per tile.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"

namespace vtm {

constexpr int kIn = VTM_MLP_IN;
constexpr int kH = VTM_MLP_HIDDEN;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;
constexpr int kTile = 128;  // samples per CTA in the gradient kernel

static_assert(kParams == VTM_MLP_PARAMS, "parameter count");

__device__ __forceinline__ void load_weights(const __nv_bfloat16* __restrict__ wb, float* w) {
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
}

__global__ void k_mlp_forward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ X, float* __restrict__ y,
                              int64_t n) {
  __shared__ float w[kParams];
  load_weights(wb, w);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x[k] = X[i * kIn + k];
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float a = w[kOffB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(w[kOffW1 + j * kIn + k], x[k], a);
    h1[j] = fmaxf(a, 0.f);
  }
  float out = w[kOffB3];
  for (int j2 = 0; j2 < kH; ++j2) {
    float a = w[kOffB2 + j2];
#pragma unroll
    for (int j = 0; j < kH; ++j) a = fmaf(w[kOffW2 + j2 * kH + j], h1[j], a);
    out = fmaf(w[kOffW3 + j2], fmaxf(a, 0.f), out);
  }
  y[i] = out;
}

// Mean-squared-error loss over n samples and its gradient w.r.t. the (BF16) weights, accumulated
// into grad (zeroed by the caller) and loss[0].
__global__ void __launch_bounds__(kTile) k_mlp_grad(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ X,
                                                   const float* __restrict__ t, int64_t n, float inv_n,
                                                   float* __restrict__ grad, float* __restrict__ loss) {
  // dynamic shared memory: weights, then per-sample rows of layer-1 activations (H1), layer-2
  // deltas (D2), layer-2 activations / layer-1 deltas (D1), inputs (XS)
  extern __shared__ float sm[];
  float* w = sm;
  float(*H1)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(sm + kParams + 3);
  float(*D2)[kH + 1] = H1 + kTile;
  float(*D1)[kH + 1] = D2 + kTile;
  float(*XS)[kIn] = reinterpret_cast<float(*)[kIn]>(D1 + kTile);
  float* DY = reinterpret_cast<float*>(XS + kTile);
  __shared__ float red[kTile / 32];
  load_weights(wb, w);
  __syncthreads();
  const int tid = threadIdx.x;
  const int64_t i = blockIdx.x * (int64_t)kTile + tid;
  const bool live = i < n;
  float x[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) {
    x[k] = live ? X[i * kIn + k] : 0.f;
    XS[tid][k] = x[k];
  }
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float a = w[kOffB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(w[kOffW1 + j * kIn + k], x[k], a);
    h1[j] = fmaxf(a, 0.f);
    H1[tid][j] = h1[j];
  }
  float out = w[kOffB3];
  for (int j2 = 0; j2 < kH; ++j2) {
    float a = w[kOffB2 + j2];
#pragma unroll
    for (int j = 0; j < kH; ++j) a = fmaf(w[kOffW2 + j2 * kH + j], h1[j], a);
    const float h2 = fmaxf(a, 0.f);
    D2[tid][j2] = (a > 0.f) ? 1.f : 0.f;  // mask, scaled below
    out = fmaf(w[kOffW3 + j2], h2, out);
    D1[tid][j2] = h2;  // layer-2 activation, kept for dW3 until the layer-1 deltas replace it
  }
  const float err = live ? out - t[i] : 0.f;
  const float dy = 2.f * err * inv_n;
  // dW3 / db3 contributions use h2 (held in D1); layer-2 deltas: dy * W3 * mask
  for (int j2 = 0; j2 < kH; ++j2) D2[tid][j2] *= dy * w[kOffW3 + j2];
  // loss
  float l = err * err * inv_n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((tid & 31) == 0) red[tid >> 5] = l;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int k = 0; k < kTile / 32; ++k) s += red[k];
    atomicAdd(loss, s);
  }
  // dW3[j2] = sum_s dy_s h2_s[j2]; db3 = sum_s dy_s
  DY[tid] = dy;
  __syncthreads();
  if (tid < kH) {
    float g = 0.f;
    for (int s2 = 0; s2 < kTile; ++s2) g += DY[s2] * D1[s2][tid];
    atomicAdd(&grad[kOffW3 + tid], g);
  } else if (tid == kH) {
    float g = 0.f;
    for (int s2 = 0; s2 < kTile; ++s2) g += DY[s2];
    atomicAdd(&grad[kOffB3], g);
  }
  __syncthreads();
  // layer-1 deltas: D1[s][j] = (sum_j2 W2[j2][j] D2[s][j2]) * [h1 > 0]
  for (int j = 0; j < kH; ++j) {
    float a = 0.f;
#pragma unroll 8
    for (int j2 = 0; j2 < kH; ++j2) a = fmaf(w[kOffW2 + j2 * kH + j], D2[tid][j2], a);
    D1[tid][j] = (h1[j] > 0.f) ? a : 0.f;
  }
  __syncthreads();
  // dW2[j2][j] = sum_s D2[s][j2] H1[s][j]  (4096 entries, 32 per thread); db2[j2] = sum_s D2[s][j2]
  for (int e = tid; e < kH * kH; e += kTile) {
    const int j2 = e / kH, j = e % kH;
    float g = 0.f;
    for (int s2 = 0; s2 < kTile; ++s2) g = fmaf(D2[s2][j2], H1[s2][j], g);
    atomicAdd(&grad[kOffW2 + e], g);
  }
  for (int e = tid; e < kH; e += kTile) {
    float g = 0.f, g1 = 0.f;
    for (int s2 = 0; s2 < kTile; ++s2) {
      g += D2[s2][e];
      g1 += D1[s2][e];
    }
    atomicAdd(&grad[kOffB2 + e], g);
    atomicAdd(&grad[kOffB1 + e], g1);
  }
  // dW1[j][k] = sum_s D1[s][j] X[s][k]
  for (int e = tid; e < kH * kIn; e += kTile) {
    const int j = e / kIn, k = e % kIn;
    float g = 0.f;
    for (int s2 = 0; s2 < kTile; ++s2) g = fmaf(D1[s2][j], XS[s2][k], g);
    atomicAdd(&grad[kOffW1 + e], g);
  }
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       __nv_bfloat16* __restrict__ wb, int np, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  wb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb, int np) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) wb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace vtm

struct vtm_mlp {
  float* p = nullptr;       // FP32 master parameters (device)
  float* m = nullptr;       // Adam first moment
  float* v = nullptr;       // Adam second moment
  float* g = nullptr;       // gradient
  float* loss = nullptr;    // device scalar
  __nv_bfloat16* wb = nullptr;  // BF16 weights used by the kernels
  int64_t step = 0;
  ~vtm_mlp() {
    cudaFree(p);
    cudaFree(m);
    cudaFree(v);
    cudaFree(g);
    cudaFree(loss);
    cudaFree(wb);
  }
};

namespace vtm {

#define MLP_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) fail(VTM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based generator for the initial weights.
static uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

static double uniform01(uint64_t seed, uint64_t k) { return (double)(splitmix64(seed * 0x100000001B3ull + k) >> 11) * 0x1.0p-53; }

vtm_mlp* mlp_create(uint64_t seed) {
  std::unique_ptr<vtm_mlp> m(new vtm_mlp());
  const size_t pb = kParams * sizeof(float);
  MLP_CUDA(cudaMalloc(&m->p, pb));
  MLP_CUDA(cudaMalloc(&m->m, pb));
  MLP_CUDA(cudaMalloc(&m->v, pb));
  MLP_CUDA(cudaMalloc(&m->g, pb));
  MLP_CUDA(cudaMalloc(&m->loss, sizeof(float)));
  MLP_CUDA(cudaMalloc(&m->wb, kParams * sizeof(__nv_bfloat16)));
  // He-uniform weights, zero biases
  std::vector<float> h(kParams, 0.f);
  auto fill = [&](int off, int rows, int cols) {
    const double a = std::sqrt(6.0 / cols);
    for (int r = 0; r < rows * cols; ++r) h[off + r] = (float)((2.0 * uniform01(seed, off + r) - 1.0) * a);
  };
  fill(kOffW1, kH, kIn);
  fill(kOffW2, kH, kH);
  fill(kOffW3, 1, kH);
  MLP_CUDA(cudaMemcpy(m->p, h.data(), pb, cudaMemcpyHostToDevice));
  MLP_CUDA(cudaMemset(m->m, 0, pb));
  MLP_CUDA(cudaMemset(m->v, 0, pb));
  MLP_CUDA(cudaMemset(m->g, 0, pb));
  k_to_bf16<<<(kParams + 255) / 256, 256>>>(m->p, m->wb, kParams);
  MLP_CUDA(cudaGetLastError());
  MLP_CUDA(cudaDeviceSynchronize());
  return m.release();
}

void mlp_set_params(vtm_mlp* m, const float* host) {
  MLP_CUDA(cudaMemcpy(m->p, host, kParams * sizeof(float), cudaMemcpyHostToDevice));
  MLP_CUDA(cudaMemset(m->m, 0, kParams * sizeof(float)));
  MLP_CUDA(cudaMemset(m->v, 0, kParams * sizeof(float)));
  m->step = 0;
  k_to_bf16<<<(kParams + 255) / 256, 256>>>(m->p, m->wb, kParams);
  MLP_CUDA(cudaGetLastError());
  MLP_CUDA(cudaDeviceSynchronize());
}

void mlp_get_params(const vtm_mlp* m, float* host) {
  MLP_CUDA(cudaMemcpy(host, m->p, kParams * sizeof(float), cudaMemcpyDeviceToHost));
}

void mlp_get_grads(const vtm_mlp* m, float* host) {
  MLP_CUDA(cudaMemcpy(host, m->g, kParams * sizeof(float), cudaMemcpyDeviceToHost));
}

void mlp_forward(const vtm_mlp* m, const float* X, float* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(m->wb, X, y, n);
  MLP_CUDA(cudaGetLastError());
}

float mlp_loss_grad(vtm_mlp* m, const float* X, const float* t, int64_t n, cudaStream_t st) {
  if (n <= 0) fail(VTM_ERR_INVALID, "empty batch");
  MLP_CUDA(cudaMemsetAsync(m->g, 0, kParams * sizeof(float), st));
  MLP_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
  const size_t smem = sizeof(float) * ((size_t)kParams + 3 + 3 * kTile * (kH + 1) + kTile * kIn + kTile);
  static bool configured = false;
  if (!configured) {
    MLP_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = true;
  }
  k_mlp_grad<<<(unsigned)((n + kTile - 1) / kTile), kTile, smem, st>>>(m->wb, X, t, n, 1.f / (float)n, m->g, m->loss);
  MLP_CUDA(cudaGetLastError());
  float l = 0.f;
  MLP_CUDA(cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
  MLP_CUDA(cudaStreamSynchronize(st));
  return l;
}

void mlp_destroy(vtm_mlp* m) { delete m; }

void mlp_adam(vtm_mlp* m, float lr, float b1, float b2, float eps, cudaStream_t st) {
  m->step++;
  const float c1 = 1.f - (float)std::pow((double)b1, (double)m->step);
  const float c2 = 1.f - (float)std::pow((double)b2, (double)m->step);
  k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(m->p, m->m, m->v, m->g, m->wb, kParams, lr, b1, b2, eps, c1, c2);
  MLP_CUDA(cudaGetLastError());
}

}  // namespace vtm
