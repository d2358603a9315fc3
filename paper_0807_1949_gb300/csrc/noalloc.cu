// vtm_relative_residual_noalloc: the FP64 relative residual ||b_r - A x_r|| / ||b_r|| without any
// device allocation.
//
// Some callers cannot allocate device memory at the moment they need this number: a monitoring
// thread of a service whose device memory is fully reserved up front by a framework's caching
// allocator (a raw cudaMalloc there can fail even though the framework still has free blocks), or
// a latency-critical loop that must not call cudaMalloc/cudaFree because they can synchronise the
// device.  For them this entry point keeps its only scratch — the per-right-hand-side sums of
// squares — in a file-scope device array that the device holds from the moment this code is
// loaded onto it until the process exits.  The caller passes every input and the output.
//
// CUDA loads a library's device code lazily by default: the array (and this file's kernel) are
// put on a device, which allocates device memory, when the first call on that device looks up the
// array's address.  vtm_setup does that look-up for its device, so a caller that built a solver
// has nothing left to load; any other caller makes one warm-up call per device before device
// memory is reserved up front (and before any stream capture).  Later calls allocate nothing.
#include <mutex>
#include <string>

#include "internal.h"
#include "kernels.h"

namespace {

// Scratch of the entry point: [0, VTM_NOALLOC_MAX_RHS) sums of squares of the residuals,
// [VTM_NOALLOC_MAX_RHS, 2*VTM_NOALLOC_MAX_RHS) sums of squares of b.  2 * 8 doubles = 128 bytes.
static __device__ __align__(256) double g_noalloc_scratch[2 * VTM_NOALLOC_MAX_RHS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// In host code the name g_noalloc_scratch is only a host-side stand-in; the kernels need the
// device address, looked up once per device with that device current.
double* scratch_for_current_device() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) vtm::fail(VTM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) vtm::fail(VTM_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      vtm::fail(VTM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}

__global__ void k_noalloc_finish(int nrhs, const double* __restrict__ sums, double* __restrict__ rel) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  const double rr = sums[r], bb = sums[VTM_NOALLOC_MAX_RHS + r];
  rel[r] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : sqrt(rr);
}

}  // namespace

namespace vtm {
// Loads the array onto the current device and caches its address (called by vtm_setup).
void noalloc_prepare_current_device() { scratch_for_current_device(); }
}  // namespace vtm

extern "C" int vtm_relative_residual_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                                             int32_t nrhs, const double* b, int64_t ldb, const double* x,
                                             int64_t ldx, double* rel, void* cuda_stream) {
  try {
    if (n <= 0 || !rowptr || !col || !val || !b || !x || !rel)
      vtm::fail(VTM_ERR_INVALID, "vtm_relative_residual_noalloc: null pointer or n <= 0");
    if (nrhs < 1 || nrhs > VTM_NOALLOC_MAX_RHS)
      vtm::fail(VTM_ERR_INVALID, "vtm_relative_residual_noalloc: nrhs must be in [1, " +
                                     std::to_string(VTM_NOALLOC_MAX_RHS) + "], got " + std::to_string(nrhs));
    if (ldb < n || ldx < n) vtm::fail(VTM_ERR_INVALID, "vtm_relative_residual_noalloc: leading dimension < n");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double* sums = scratch_for_current_device();
    // the array keeps the previous call's sums: clear both halves before accumulating
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * VTM_NOALLOC_MAX_RHS * sizeof(double), st);
    if (e == cudaSuccess) e = vtm::launch_sqnorm(n, nrhs, b, ldb, sums + VTM_NOALLOC_MAX_RHS, st);
    if (e == cudaSuccess)
      e = vtm::launch_residual(n, nrhs, rowptr, col, val, b, ldb, x, ldx, nullptr, 0, sums, st);
    if (e == cudaSuccess) {
      k_noalloc_finish<<<1, 32, 0, st>>>(nrhs, sums, rel);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess)
      vtm::fail(VTM_ERR_CUDA, std::string("vtm_relative_residual_noalloc: ") + cudaGetErrorString(e));
    return VTM_OK;
  } catch (const vtm::Error& err) {
    vtm::set_last_error(err.msg);
    return err.code;
  } catch (...) {
    vtm::set_last_error("vtm_relative_residual_noalloc: unexpected error");
    return VTM_ERR_INVALID;
  }
}
