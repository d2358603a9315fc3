// One VTM sweep for 16 or 32 right-hand sides with the band products on the tensor cores (Table 1
// steps 3-5, eq. 5.6 / 5.8 per column; the same sweep as sweep_wide.cu).
//
// Factor.  Row i of the subgraph's factor L (K_j = L L^T, eq. 5.8) is scaled by d_i = 1 / ||L_i||_2
// (the rows of D^-1/2 L, D = diag(K_j), have unit norm, so every entry lies in [-1, 1]); the sweep
// solves (D^-1/2 L)(D^-1/2 L)^T x~ = D^-1/2 r and returns x = D^-1/2 x~.  Rows go in groups of
// 128.  Group g (rows k0 = 128 g ..) keeps two operands, each as fp16 pairs hi = fp16(v),
// lo = fp16(2^11 (v - hi)) (about 22 significant bits together, lo a normal fp16 number down to
// |v| ~ 2^-14) in 128 x 64 panels of the 128-byte-swizzled K-major layout of tcgen05:
//  * the entries left of the group, columns k0 - 128 T .. k0 - 1 (T = ceil(w / 128) tiles, w the
//    half-bandwidth): 2 T panels, of which the first is left out when it lies entirely left of the
//    band (w <= 128 T - 64; its products are zero);
//  * the inverse of the group's 128 x 128 diagonal block, G_g = inv(L~_gg) (lower triangular; the
//    balanced factor keeps its entries of order one): 2 panels.
//
// Forward pass, group by group: t = r~_g - L~_(g, left) y_left (M = 128, N = R, K = 128 T), then
// y_g = G_g t (K = 128).  Backward pass, groups in descending order: x~_g = G_g^T t with
// t = y~_g minus what the later groups have added to the group's accumulator, then
// L~_(g, left)^T x~_g (the same panels read MN-major: M = 128 rows of one tile, K = the group's 128
// rows) adds to the accumulators of the T groups to its left; group h collects the contributions
// of groups h + 1 .. h + T in one tensor-memory accumulator, which it reads once.  G_g^T is G_g's
// panels read MN-major.  Every product is three fp16 products per K step with FP32 accumulation in
// tensor memory: hi hi into one accumulator, hi lo + lo hi into a second one scaled back by 2^-11.
// The vector operands (the window of y, t, x~) are fp16 hi / lo of v / sigma, sigma a power of two
// per column at or above max |r~| (forward) or max |y~| (backward).
//
// Warps: 0 streams the panels through a ring of 16 KB slots (bulk copies, one panel each), 1 issues
// the MMAs, 3-10 move the vectors (256 threads, thread = one row of the group and half of the
// columns: the tensor-memory loads, the fp16 operands, the results).  The forward left product has
// two tensor-memory buffers, so that the part of group g + 1's product that does not need y_g runs
// while the SIMT warps finish group g.  Every wait is bounded; a CTA that gives up
// records VTM_ERR_TIMEOUT, lets its copies and MMAs finish, frees its tensor memory and returns.
#include "kernels.h"
#include "tc.cuh"

namespace vtm {

using namespace tc;

namespace {

constexpr int kG = 128;                              // rows per group (MMA M)
constexpr int kMaxT = kWideTcMaxTiles;               // tiles left of a group (half-bandwidth <= 384)
constexpr int kNWC = 2 * kMaxT;                      // 64-row chunks of the forward window
constexpr int kSimtWarps = 8;
constexpr int kWtThreads = 32 * (3 + kSimtWarps);
constexpr int kSimtThreads = 32 * kSimtWarps;
constexpr int kSimtBar = 1;
constexpr uint32_t kChunk = 16384;                   // one fp16 panel: 128 rows x 64 columns (a ring slot)
constexpr uint32_t kZeroBytes = kChunk;              // a zero panel at the start of the factor buffer
constexpr uint32_t kDBytes = 512;                    // the group's 128 row scales d_i
constexpr float kLoScale = 2048.f;                   // lo halves are stored times 2^11

// Group layout, z = 1 when the first left panel is left out (w <= 128 T - 64), nl = 2 T - z:
// [hi of left panels z .. 2 T - 1][lo of them][hi of G_g (2 panels)][lo of G_g][d]
__host__ __device__ __forceinline__ int wt_tiles(int w) { return w <= 0 ? 1 : (w + kG - 1) / kG; }
__host__ __device__ __forceinline__ int wt_zlead(int w) { return (w <= kG * wt_tiles(w) - 64) ? 1 : 0; }
__host__ __device__ __forceinline__ int wt_nleft(int w) { return 2 * wt_tiles(w) - wt_zlead(w); }
__host__ __device__ __forceinline__ int64_t wt_group_bytes(int w) { return (2LL * wt_nleft(w) + 4) * kChunk + kDBytes; }
__host__ __device__ __forceinline__ int wt_groups(int n) { return (n + kG - 1) / kG; }

template <int R>
struct WtLayout {
  static constexpr uint32_t kWinChunk = 256u * R;    // hi + lo panels (R rows x 128 bytes each)
  // ring slots: what the 227 KB leave after the window, the t operand and 2 KB of barriers, even;
  // at R = 32 eight of the ten that fit (each slot given up goes to the L1 cache the vector warps'
  // gathers hit in; measured per sweep at 256^3 x 32: 6 / 8 / 10 slots 16.7 / 15.1 / 15.4 ms)
  static constexpr int kFit = (int)((232448u - 2048u - (kNWC + 2) * kWinChunk) / kChunk) & ~1;
  static constexpr int kSlots = R == 32 ? (kFit < 8 ? kFit : 8) : kFit;
  static constexpr uint32_t kWin = kSlots * kChunk;             // forward window (backward: x~)
  static constexpr uint32_t kB2 = kWin + kNWC * kWinChunk;      // t of the group (K = 128)
  static constexpr uint32_t kEnd = kB2 + 2 * kWinChunk;
  static constexpr uint32_t kBytes = 1024 + 1024 + kEnd;        // alignment slack + barrier page
  static_assert(kBytes <= 232448u, "shared memory");
};

__device__ __forceinline__ void simt_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(kSimtBar), "n"(kSimtThreads) : "memory");
}

// Bounded wait that also gives up once another role has set the abort flag.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, long limit, volatile int* abort_flag) {
  if (mbar_test_wait(bar, parity)) return true;  // most waits find the phase complete
  for (long it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ float pow2_at_or_above(float m) {
  int e = 0;
  if (!(m > 0.f) || !isfinite(m)) return 1.f;
  frexpf(m, &e);
  return ldexpf(1.f, e);
}

__device__ __forceinline__ void split_store(unsigned char* hi_panel, unsigned char* lo_panel, uint32_t off, float v) {
  const __half h = __float2half_rn(v);
  *reinterpret_cast<__half*>(hi_panel + off) = h;
  *reinterpret_cast<__half*>(lo_panel + off) = __float2half_rn((v - __half2float(h)) * kLoScale);
}

// Dynamic shared memory of the factor kernel: G_g (128 x kXs), one block row of L~_gg (32 x 97) and
// a 32 x 33 product.
constexpr int kXs = 132;
constexpr size_t kFactorSmem = (size_t)(kG * kXs + 32 * 97 + 32 * 33) * sizeof(float);

}  // namespace

int64_t wide_tc_bytes(int n, int w) { return (int64_t)wt_groups(n) * wt_group_bytes(w); }
int64_t wide_tc_zero_bytes() { return kZeroBytes; }
bool wide_tc_fits(int w) { return wt_tiles(w) <= kMaxT; }
int wide_tc_groups(int n) { return wt_groups(n); }

size_t wide_tc_smem_bytes(int R) { return R == 16 ? WtLayout<16>::kBytes : WtLayout<32>::kBytes; }

// The tensor-core factor of group blockIdx.y of subgraph blockIdx.x from its FP32 band factor (whose
// 32 x 32 diagonal blocks hold the inverses of the Cholesky blocks).  Rows past the band storage
// (n_pad .. 128 ng) are identity rows.  G_g by block forward substitution over the four 32-row
// blocks: G_ii = inv(L~_ii), G_ij = -G_ii sum_{k=j}^{i-1} L~_ik G_kj.
__global__ void __launch_bounds__(256) k_wide_tc_factor(const PieceDesc* __restrict__ pieces, const float* __restrict__ band,
                                                         unsigned char* __restrict__ wt) {
  const PieceDesc pd = pieces[blockIdx.x];
  const int g = blockIdx.y;
  if (g >= wt_groups(pd.n)) return;
  const int T = wt_tiles(pd.w), z = wt_zlead(pd.w), nl = wt_nleft(pd.w), Wp = pd.Wp, off = Wp - 1, k0 = g * kG;
  unsigned char* gb = wt + pd.wt_off + (int64_t)g * wt_group_bytes(pd.w);
  const float* L = band + pd.factor_off;
  extern __shared__ float fsm[];
  float* X = fsm;                 // G_g, [128][kXs]
  float* lt = X + kG * kXs;       // block row i of L~_gg left of its diagonal block, [32][97]
  float* pb = lt + 32 * 97;       // [32][33]
  __shared__ float inv[4][32][33];  // stored inverse diagonal blocks
  __shared__ float lkk[4][32][33];  // the Cholesky blocks recovered from them (for the row norms)
  __shared__ float dsh[kG];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto entry = [&](int row, int col) -> float {  // L[row][col] inside the band storage, else 0
    if (row >= pd.n_pad || col < 0 || col < row - off || col > row) return 0.f;
    return L[(int64_t)row * Wp + (col - row + off)];
  };
  for (int e = tid; e < 4 * 32 * 32; e += blockDim.x) {
    const int b = e >> 10, r = (e >> 5) & 31, c = e & 31;
    const int row = k0 + 32 * b + r;
    float v;
    if (row >= pd.n_pad) v = (r == c) ? 1.f : 0.f;
    else v = (c <= r) ? entry(row, k0 + 32 * b + c) : 0.f;
    inv[b][r][c] = v;
  }
  for (int e = tid; e < kG * kXs; e += blockDim.x) X[e] = 0.f;
  __syncthreads();
  if (warp < 4) {
    // solve inv * X = I column by column (lane = column j): X = L_KK, lower triangular
    const int b = warp, j = lane;
    for (int i = 0; i < 32; ++i) {
      if (i < j) {
        lkk[b][i][j] = 0.f;
        continue;
      }
      float s = (i == j) ? 1.f : 0.f;
      for (int k = j; k < i; ++k) s -= inv[b][i][k] * lkk[b][k][j];
      lkk[b][i][j] = s / inv[b][i][i];
    }
  }
  __syncthreads();
  if (tid < kG) {
    const int row = k0 + tid;
    float s = 1.f;
    if (row < pd.n_pad) {
      const int b = tid >> 5, r = tid & 31;
      s = 0.f;
      for (int c = 0; c <= r; ++c) s += lkk[b][r][c] * lkk[b][r][c];
      const int cb = row - (row & 31);
      for (int col = max(0, row - off); col < cb; ++col) {
        const float v = entry(row, col);
        s += v * v;
      }
    }
    dsh[tid] = s > 0.f ? rsqrtf(s) : 1.f;
  }
  __syncthreads();
  // G_ii = inv(D^-1/2 L_ii) = inv(L_ii) D^1/2
  for (int e = tid; e < 4 * 32 * 32; e += blockDim.x) {
    const int b = e >> 10, r = (e >> 5) & 31, c = e & 31;
    X[(32 * b + r) * kXs + 32 * b + c] = inv[b][r][c] / dsh[32 * b + c];
  }
  __syncthreads();
  const int pr = tid >> 3, pc = (tid & 7) * 4;  // this thread's 4 entries of a 32 x 32 block
  for (int i = 1; i < 4; ++i) {
    for (int e = tid; e < 32 * 32 * i; e += blockDim.x) {
      const int r = e / (32 * i), m = e % (32 * i);
      lt[r * 97 + m] = entry(k0 + 32 * i + r, k0 + m) * dsh[32 * i + r];
    }
    __syncthreads();
    for (int j = i - 1; j >= 0; --j) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int m = 32 * j; m < 32 * i; ++m) {
        const float l = lt[pr * 97 + m];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(l, X[m * kXs + 32 * j + pc + u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) pb[pr * 33 + pc + u] = acc[u];
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = 0.f;
      for (int m = 0; m < 32; ++m) {
        const float gm = X[(32 * i + pr) * kXs + 32 * i + m];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(gm, pb[m * 33 + pc + u], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) X[(32 * i + pr) * kXs + 32 * j + pc + u] = -acc[u];
      __syncthreads();
    }
  }
  // panels of G_g: columns 64 c .. 64 c + 63 in panel c
  for (int e = tid; e < kG * kG; e += blockDim.x) {
    const int r = e >> 7, c = e & 127;
    split_store(gb + (size_t)(2 * nl + (c >> 6)) * kChunk, gb + (size_t)(2 * nl + 2 + (c >> 6)) * kChunk,
                swz16(r, c & 63), X[r * kXs + c]);
  }
  // the left panels: panel c (c = z .. 2 T - 1) covers columns k0 - 128 T + 64 c .. + 63
  for (int e = tid; e < nl * kG * 64; e += blockDim.x) {
    const int c = z + e / (kG * 64), r = (e >> 6) & (kG - 1), kk = e & 63;
    const int row = k0 + r, col = k0 - kG * T + 64 * c + kk;
    split_store(gb + (size_t)(c - z) * kChunk, gb + (size_t)(nl + c - z) * kChunk, swz16(r, kk),
                entry(row, col) * dsh[r]);
  }
  float* dd = reinterpret_cast<float*>(gb + (size_t)(2 * nl + 4) * kChunk);
  if (tid < kG) dd[tid] = dsh[tid];
}

template <int R>
__global__ void __launch_bounds__(kWtThreads, 1) k_sweep_wide_tc(const SweepArgs<float, float> a) {
  using LY = WtLayout<R>;
  constexpr int kSlots = LY::kSlots;
  constexpr int kHalf = R / 2;            // columns of a SIMT thread (row = tensor-memory lane)
  constexpr uint32_t idK = idesc_f16(false, R), idT = idesc_f16(true, R);
  // N = 2R: the hi and lo panels of a vector operand lie one after the other (R rows of 128 bytes
  // each), so hi(A) [v_hi | v_lo] is one MMA into the accumulator pair D1 | D2
  constexpr uint32_t idK2 = idesc_f16(false, 2 * R), idT2 = idesc_f16(true, 2 * R);
  // Tensor memory.  Consecutive MMAs into one accumulator wait for each other, so every product
  // alternates its K steps between two accumulator sets (summed when read); a set is D1 | D2 (2R
  // columns).  Forward: [0, 8R) the left products of groups g even / odd, [8R, 12R) the product with
  // G_g.  Backward: [0, 12R) the accumulators of three groups (h mod 3: a group receives from the
  // T <= 3 groups after it), [12R, 16R) the product with G_g^T.
  constexpr uint32_t kTmemCols = 16 * R;
  constexpr uint32_t kSet = 2 * R;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm);
  uint64_t* full = bars;                 // [kSlots] ring slots landed
  uint64_t* empty = bars + kSlots;       // [kSlots] MMAs done with the slot
  uint64_t* accfull = bars + 2 * kSlots;      // forward: left product of the group complete
  uint64_t* bready = accfull + 1;        // forward: the group's y is in the window
  uint64_t* tready = accfull + 2;        // the group's t operand is written (both passes)
  uint64_t* yready = accfull + 3;        // the product with G_g is complete (both passes)
  uint64_t* baccready = accfull + 4;     // backward: the next group's accumulator is complete
  uint64_t* xready = accfull + 5;        // backward: the group's x~ operand is written
  uint64_t* xfree = accfull + 6;         // backward: the MMAs are done with that operand
  uint64_t* done = accfull + 7;          // every MMA has completed
  const int kBars = 2 * kSlots + 8;
  volatile int* flags = reinterpret_cast<volatile int*>(bars + kBars);  // [0] abort, [1] SIMT decision
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kBars + 2);
  static_assert(8 * (2 * kSlots + 8) + 16 <= 384, "barrier page");
  float* sigf = reinterpret_cast<float*>(sm + 384);  // [R] forward operand scale per column
  float* sigb = sigf + 32;                           // [R] backward
  const uint32_t regA = base + 1024;
  unsigned char* pA = sm + 1024;
  float* scr = reinterpret_cast<float*>(pA + LY::kB2);  // [8][R / 2] column maxima (t operand is free then)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int n = pd.n, T = wt_tiles(pd.w), z = wt_zlead(pd.w), nl = wt_nleft(pd.w), ng = wt_groups(n);
  const int64_t GB = wt_group_bytes(pd.w);
  const unsigned char* gb0 = a.wt + pd.wt_off;
  const unsigned char* zero_panel = a.wt;  // the factor buffer starts with a zero panel
  float* xg = a.xc + (size_t)pd.copy_off * R;
  const float* bg = a.bt + (size_t)pd.copy_off * R;
  auto dval = [&](int row) -> float {
    return *reinterpret_cast<const float*>(gb0 + (int64_t)(row / kG) * GB + (size_t)(2 * nl + 4) * kChunk +
                                           (size_t)(row % kG) * 4);
  };
  // left panel c (hi, or lo with lo = 1) of group g; c < z: the zero panel
  auto left_panel = [&](int g, int c, int lo) -> const unsigned char* {
    if (c < z) return zero_panel;
    return gb0 + (int64_t)g * GB + (size_t)(lo * nl + c - z) * kChunk;
  };

  if (tid == 0) {
    for (int i = 0; i < kBars; ++i) mbar_init(&bars[i], 1);
    flags[0] = 0;
    flags[1] = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // ---- r~ = D^-1/2 (b~ + P (Y w_in)) (port currents from the twins' waves) into xc, and the column
  // maxima of r~ (a port row also counts with its value before the currents: sigma only has to be
  // at or above max |r~|)
  {
    float mx[4] = {0.f, 0.f, 0.f, 0.f};  // columns 4 (tid % (R / 4)) .. + 3 (kWtThreads is a multiple of R / 4)
    const float4* b4 = reinterpret_cast<const float4*>(bg);
    float4* x4 = reinterpret_cast<float4*>(xg);
    constexpr int kU = 4;
    for (int i0 = tid; i0 < n * (R / 4); i0 += kWtThreads * kU) {
      float4 v[kU];
      float dv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * kWtThreads;
        v[u] = i < n * (R / 4) ? b4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        dv[u] = i < n * (R / 4) ? dval(i / (R / 4)) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * kWtThreads;
        if (i < n * (R / 4)) {
          const float4 o = make_float4(v[u].x * dv[u], v[u].y * dv[u], v[u].z * dv[u], v[u].w * dv[u]);
          x4[i] = o;
          mx[0] = fmaxf(mx[0], fabsf(o.x)), mx[1] = fmaxf(mx[1], fabsf(o.y));
          mx[2] = fmaxf(mx[2], fabsf(o.z)), mx[3] = fmaxf(mx[3], fabsf(o.w));
        }
      }
    }
    __syncthreads();
    // port rows, one port per thread with its R columns in registers (16-byte loads of the R-wide
    // wave rows): r~ += d_row (sum_e w_in[e] / Z_e + coupling currents)
    float mp[R];
#pragma unroll
    for (int c = 0; c < R; ++c) mp[c] = 0.f;
    for (int q = tid; q < pd.nports; q += kWtThreads) {
      const int port = pd.port_off + q;
      float acc[R];
#pragma unroll
      for (int c = 0; c < R; ++c) acc[c] = 0.f;
      for (int e = a.port_end_ptr[port]; e < a.port_end_ptr[port + 1]; ++e) {
        const float4* w = reinterpret_cast<const float4*>(a.wprev + (size_t)a.twin[e] * R);
        const float iz = a.invz[e];
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          const float4 x = w[k4];
          acc[4 * k4] += x.x * iz, acc[4 * k4 + 1] += x.y * iz, acc[4 * k4 + 2] += x.z * iz, acc[4 * k4 + 3] += x.w * iz;
        }
      }
      if (a.cpl.ptr)
        for (int k = a.cpl.ptr[port]; k < a.cpl.ptr[port + 1]; ++k) {
          const float yk = a.cpl.y[k];
          const float4* w = reinterpret_cast<const float4*>(a.wprev + (size_t)a.cpl.oth[k] * R);
#pragma unroll
          for (int k4 = 0; k4 < R / 4; ++k4) {
            const float4 x = w[k4];
            acc[4 * k4] += yk * x.x, acc[4 * k4 + 1] += yk * x.y, acc[4 * k4 + 2] += yk * x.z, acc[4 * k4 + 3] += yk * x.w;
          }
        }
      const int row = a.port_local[port];
      const float dv = dval(row);
      float4* xr = reinterpret_cast<float4*>(xg + (size_t)row * R);
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) {
        float4 x = xr[k4];
        x.x += dv * acc[4 * k4], x.y += dv * acc[4 * k4 + 1], x.z += dv * acc[4 * k4 + 2], x.w += dv * acc[4 * k4 + 3];
        xr[k4] = x;
        mp[4 * k4] = fmaxf(mp[4 * k4], fabsf(x.x)), mp[4 * k4 + 1] = fmaxf(mp[4 * k4 + 1], fabsf(x.y));
        mp[4 * k4 + 2] = fmaxf(mp[4 * k4 + 2], fabsf(x.z)), mp[4 * k4 + 3] = fmaxf(mp[4 * k4 + 3], fabsf(x.w));
      }
    }
    // per column: the 4-wide maxima of the threads with tid % (R / 4) == c / 4, and every thread's
    // port-row maximum
    float* red = reinterpret_cast<float*>(pA + LY::kWin);  // the window, zeroed below
    reinterpret_cast<float4*>(red)[tid] = make_float4(mx[0], mx[1], mx[2], mx[3]);
#pragma unroll
    for (int c = 0; c < R; ++c) red[4 * kWtThreads + c * kWtThreads + tid] = mp[c];
    __syncthreads();
    if (tid < R) {
      float m = 0.f;
      for (int t = tid / 4; t < kWtThreads; t += R / 4) m = fmaxf(m, red[4 * t + (tid & 3)]);
      for (int t = 0; t < kWtThreads; ++t) m = fmaxf(m, red[4 * kWtThreads + tid * kWtThreads + t]);
      sigf[tid] = pow2_at_or_above(m);
    }
    __syncthreads();
    // the forward window starts as zeros (the columns left of row 0)
    uint4* win = reinterpret_cast<uint4*>(pA + LY::kWin);
    for (int i = tid; i < (int)(kNWC * LY::kWinChunk / 16); i += kWtThreads) win[i] = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  const uint32_t tmem = *tslot;

  // Order of the panels (the MMA issuer takes them in the same order).  Forward: group 0's left
  // panels, then per group g: the left panels of group g + 1 that do not read y_g ("early"), G_g's
  // hi and lo pairs, the two that do ("late").  Backward, per group in descending order: G_g's pairs,
  // then the hi and lo pairs of tiles T - 1 .. 0 (tiles left of row 0 skipped).  A left panel is its
  // hi then its lo half; left panels c < z are not stored (or read) forward and come from the zero
  // panel backward.
  const int nearly = 2 * T - 2;  // left panels of a group that do not read the previous group's y

  if (warp == 0) {
    // ---- panels: one 16 KB bulk copy per slot, read once per pass (evict first)
    if (lane == 0) {
      uint64_t pol;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
      int cnt = 0;
      bool ok = true;
      auto next = [&](const unsigned char* src) {
        if (!ok) return;
        const int slot = cnt % kSlots;
        if (cnt >= kSlots && !wait_or_abort(&empty[slot], (uint32_t)(((cnt / kSlots) - 1) & 1), a.wait_limit, flags)) {
          ok = false;
          return;
        }
        if (cnt != a.withhold) {  // testing hook: this copy's wait can only run out
          mbar_arrive_expect_tx(&full[slot], kChunk);
          bulk_g2s_hint(regA + slot * kChunk, src, kChunk, &full[slot], pol);
        }
        ++cnt;
      };
      auto left = [&](int g, int c0, int c1) {
        for (int c = (c0 > z ? c0 : z); c < c1; ++c) {
          next(left_panel(g, c, 0));
          next(left_panel(g, c, 1));
        }
      };
      auto gpanels = [&](int g) {
        const unsigned char* src = gb0 + (int64_t)g * GB + (size_t)(2 * nl) * kChunk;
        for (int i = 0; i < 4; ++i) next(src + (size_t)i * kChunk);
      };
      left(0, 0, 2 * T);
      for (int g = 0; g < ng && ok && !flags[0]; ++g) {
        if (g + 1 < ng) left(g + 1, 0, nearly);
        gpanels(g);
        if (g + 1 < ng) left(g + 1, nearly, 2 * T);
      }
      for (int k = 0; k < ng && ok && !flags[0]; ++k) {
        const int g = ng - 1 - k;
        gpanels(g);
        for (int m = T - 1; m >= 0 && ok; --m) {
          if (g - T + m < 0) continue;
          next(left_panel(g, 2 * m, 0));
          next(left_panel(g, 2 * m + 1, 0));
          next(left_panel(g, 2 * m, 1));
          next(left_panel(g, 2 * m + 1, 1));
        }
      }
      if (!ok) flags[0] = 1;
      // copies still in flight must land before the shared memory can go away
      for (int c = (cnt > kSlots ? cnt - kSlots : 0); c < cnt; ++c)
        if (c != a.withhold) mbar_wait_bounded(&full[c % kSlots], (uint32_t)((c / kSlots) & 1), kDrainPolls);
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      int cnt = 0;
      bool ok = true;
      const uint32_t dGf = tmem + 8 * R, dGb = tmem + 12 * R;
      const uint32_t b2 = regA + LY::kB2, xb = regA + LY::kWin;
      auto take = [&]() -> uint32_t {  // the next slot's address, 0 if the wait gave up
        const int slot = cnt % kSlots;
        if (!wait_or_abort(&full[slot], (uint32_t)((cnt / kSlots) & 1), a.wait_limit, flags)) {
          ok = false;
          return 0u;
        }
        tc_fence_after();
        return regA + slot * kChunk;
      };
      auto give = [&](int k) {  // the last k slots taken are free once the MMAs issued so far complete
        for (int i = 0; i < k; ++i) mma_commit(&empty[(cnt + i) % kSlots]);
        cnt += k;
      };
      // left panels c0 .. c1 - 1 of group g into the accumulator pair at d (first issued one
      // overwrites when first is set); window rows of group g - T + c / 2
      auto left_product = [&](int g, int c0, int c1, uint32_t d, bool first) {
        int ks = 0;  // K steps issued by this call: set ks & 1, the first step of a set overwrites
        for (int c = (c0 > z ? c0 : z); c < c1 && ok; ++c) {
          const uint32_t sh = take();
          if (!ok) return;
          const uint32_t sl = regA + ((cnt + 1) % kSlots) * kChunk;
          {
            const int slot = (cnt + 1) % kSlots;
            if (!(ok = wait_or_abort(&full[slot], (uint32_t)(((cnt + 1) / kSlots) & 1), a.wait_limit, flags))) return;
            tc_fence_after();
          }
          const int gr = g - T + (c >> 1);
          const int wc = ((2 * gr + (c & 1)) % kNWC + kNWC) % kNWC;
          const uint64_t aH = sdesc(sh, 16, 1024), aL = sdesc(sl, 16, 1024);
          const uint64_t bH = sdesc(regA + LY::kWin + wc * LY::kWinChunk, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk, ++ks) {
            const uint32_t o = 2 * kk;  // 32 bytes per K step of 16
            const uint32_t ds = d + (uint32_t)(ks & 1) * kSet;
            mma_f16(ds, aH + o, bH + o, idK2, (first && ks < 2) ? 0u : 1u);
            mma_f16_acc(ds + R, aL + o, bH + o, idK);
          }
          give(2);
        }
      };
      // the product with G_g (forward) or G_g^T (backward) of the t operand, into the sets at dG
      auto g_product = [&](bool transposed, uint32_t dG) {
        const uint32_t id = transposed ? idT : idK, id2 = transposed ? idT2 : idK2;
        const uint32_t h0 = take();
        if (!ok) return;
        uint32_t slots[4] = {h0, 0u, 0u, 0u};
        for (int i = 1; i < 4; ++i) {
          const int slot = (cnt + i) % kSlots;
          if (!(ok = wait_or_abort(&full[slot], (uint32_t)(((cnt + i) / kSlots) & 1), a.wait_limit, flags))) return;
          slots[i] = regA + slot * kChunk;
        }
        tc_fence_after();
        // hi panels 0, 1 in slots 0, 1 (adjacent: the ring has an even slot count and every pair
        // starts at an even slot), lo panels in slots 2, 3
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint32_t p = kk >> 2, o = (kk & 3) * 2;
          const uint64_t ah = transposed ? sdesc(slots[0], kChunk, 1024) + (uint64_t)(kk * 128)
                                         : sdesc(slots[p], 16, 1024) + o;
          const uint64_t al = transposed ? sdesc(slots[2], kChunk, 1024) + (uint64_t)(kk * 128)
                                         : sdesc(slots[2 + p], 16, 1024) + o;
          const uint64_t bH = sdesc(b2 + p * LY::kWinChunk, 16, 1024) + o;
          const uint32_t ds = dG + (uint32_t)(kk & 1) * kSet;
          mma_f16(ds, ah, bH, id2, kk < 2 ? 0u : 1u);
          mma_f16_acc(ds + R, al, bH, id);
        }
        give(4);
        mma_commit(yready);
      };
      // forward
      left_product(0, 0, 2 * T, tmem, true);
      if (ok) mma_commit(accfull);
      for (int g = 0; g < ng && ok; ++g) {
        const uint32_t dn = tmem + (uint32_t)(((g + 1) & 1) * 2 * kSet);
        if (g + 1 < ng) left_product(g + 1, 0, nearly, dn, true);
        if (!ok) break;
        if (!(ok = wait_or_abort(tready, (uint32_t)(g & 1), a.wait_limit, flags))) break;
        tc_fence_after();
        g_product(false, dGf);
        if (!ok || g + 1 >= ng) break;
        if (!(ok = wait_or_abort(bready, (uint32_t)(g & 1), a.wait_limit, flags))) break;
        tc_fence_after();
        left_product(g + 1, nearly, 2 * T, dn, nearly <= z);
        if (ok) mma_commit(accfull);
      }
      // backward: x~_g = G_g^T t, then group g adds L~_(g, left)^T x~_g to the accumulators of
      // groups g - T .. g - 1 (tile T - 1 first: group g - 1 reads its accumulator next)
      for (int k = 0; k < ng && ok; ++k) {
        const int g = ng - 1 - k;
        if (!(ok = wait_or_abort(tready, (uint32_t)((ng + k) & 1), a.wait_limit, flags))) break;
        tc_fence_after();
        g_product(true, dGb);
        if (!ok) break;
        if (!(ok = wait_or_abort(xready, (uint32_t)(k & 1), a.wait_limit, flags))) break;
        tc_fence_after();
        for (int m = T - 1; m >= 0 && ok; --m) {
          const int h = g - T + m;
          if (h < 0) continue;
          const uint32_t d = tmem + (uint32_t)((h % 3) * 2 * kSet);
          const bool first = (g == min(h + T, ng - 1));
          const uint32_t s0 = take();
          if (!ok) break;
          for (int i = 1; i < 4 && ok; ++i) {
            const int slot = (cnt + i) % kSlots;
            ok = wait_or_abort(&full[slot], (uint32_t)(((cnt + i) / kSlots) & 1), a.wait_limit, flags);
          }
          if (!ok) break;
          tc_fence_after();
          const uint32_t s2 = regA + ((cnt + 2) % kSlots) * kChunk;
          const uint64_t aT = sdesc(s0, kChunk, 1024), aTl = sdesc(s2, kChunk, 1024);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint32_t p = kk >> 2, o = (kk & 3) * 2;
            const uint64_t bH = sdesc(xb + p * LY::kWinChunk, 16, 1024) + o;
            const uint32_t ds = d + (uint32_t)(kk & 1) * kSet;
            mma_f16(ds, aT + (uint64_t)(kk * 128), bH, idT2, (first && kk < 2) ? 0u : 1u);  // 16 rows of 128 bytes per K step
            mma_f16_acc(ds + R, aTl + (uint64_t)(kk * 128), bH, idT);
          }
          give(4);
          if (m == T - 1) mma_commit(baccready);
        }
        if (ok) mma_commit(xfree);
      }
      if (!ok) flags[0] = 1;
      mma_commit(done);  // arrives once every MMA issued above has completed
    }
  } else if (warp >= 3) {
    // ---- SIMT warps: thread = row rq of the group (tensor-memory lane), columns c0 .. c0 + R/2 - 1
    const int st = tid - 96;
    const int q = warp & 3;
    const int half = (warp - 3) >> 2;
    const int rq = 32 * q + lane;
    const int c0 = half * kHalf;
    const uint32_t tl = (uint32_t)(32 * q) << 16;
    unsigned char* b2p = pA + LY::kB2;
    auto decide = [&](uint64_t* bar, uint32_t parity) -> bool {
      if (st == 0) flags[1] = wait_or_abort(bar, parity, a.wait_limit, flags) ? 0 : 1;
      simt_sync();
      const bool ok = flags[1] == 0;
      simt_sync();
      if (!ok && st == 0) flags[0] = 1;
      return ok;
    };
    auto load_rows = [&](int g, float (&v)[kHalf]) {
      const int row = g * kG + rq;
      const bool in = g >= 0 && row < n;
      const float4* src = reinterpret_cast<const float4*>(xg + (size_t)(in ? row : 0) * R + c0);
#pragma unroll
      for (int c4 = 0; c4 < kHalf / 4; ++c4) {
        const float4 x = in ? src[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * c4] = x.x, v[4 * c4 + 1] = x.y, v[4 * c4 + 2] = x.z, v[4 * c4 + 3] = x.w;
      }
    };
    // v = D1 + 2^-11 D2 of the two accumulator sets at tensor-memory column col
    auto tmem_pair = [&](uint32_t col, float (&v)[kHalf]) {
      uint32_t a1[kHalf], a2[kHalf], b1[kHalf], b2[kHalf];
      tmem_ld<kHalf>(tmem + tl + col + c0, a1);
      tmem_ld<kHalf>(tmem + tl + col + R + c0, a2);
      tmem_ld<kHalf>(tmem + tl + col + kSet + c0, b1);
      tmem_ld<kHalf>(tmem + tl + col + kSet + R + c0, b2);
#pragma unroll
      for (int c = 0; c < kHalf; ++c)
        v[c] = (__uint_as_float(a1[c]) + __uint_as_float(b1[c])) +
               (__uint_as_float(a2[c]) + __uint_as_float(b2[c])) * (1.f / kLoScale);
    };
    // fp16 hi / lo of v / sigma as row rq of a K-major operand (K = the row in the group, panel row
    // = column)
    // (sigma is a power of two: multiplying by its reciprocal is exact)
    auto put_operand = [&](unsigned char* chunk0, const float (&v)[kHalf], const float (&sinv)[kHalf]) {
      unsigned char* pan = chunk0 + (rq >> 6) * LY::kWinChunk;
      const uint32_t kc = (uint32_t)(rq & 63) * 2;  // byte of this row (K) inside a 128-byte panel row
#pragma unroll
      for (int c = 0; c < kHalf; ++c) {
        const uint32_t n = (uint32_t)(c0 + c);
        const uint32_t off = (n >> 3) * 1024 + (n & 7) * 128 + ((((kc >> 4) ^ (n & 7))) << 4) + (kc & 15);
        split_store(pan, pan + R * 128, off, v[c] * sinv[c]);
      }
    };
    float cmax[kHalf], sg[kHalf], sinv[kHalf];
#pragma unroll
    for (int c = 0; c < kHalf; ++c) {
      cmax[c] = 0.f;
      sg[c] = sigf[c0 + c];
      sinv[c] = 1.f / sg[c];
    }
    bool ok = true;
    float rv[kHalf];
    load_rows(0, rv);
    // forward
    for (int g = 0; g < ng && ok; ++g) {
      if (!(ok = decide(accfull, (uint32_t)(g & 1)))) break;
      tc_fence_after();
      float t[kHalf];
      tmem_pair((uint32_t)((g & 1) * 2 * kSet), t);
#pragma unroll
      for (int c = 0; c < kHalf; ++c) t[c] = rv[c] - sg[c] * t[c];
      put_operand(b2p, t, sinv);
      fence_proxy_async_smem();
      tc_fence_before();
      simt_sync();
      if (st == 0) mbar_arrive(tready);
      load_rows(g + 1 < ng ? g + 1 : -1, rv);
      if (!(ok = decide(yready, (uint32_t)(g & 1)))) break;
      tc_fence_after();
      float y[kHalf];
      tmem_pair(8 * R, y);
#pragma unroll
      for (int c = 0; c < kHalf; ++c) {
        y[c] *= sg[c];
        cmax[c] = fmaxf(cmax[c], fabsf(y[c]));
      }
      const int row = g * kG + rq;
      if (row < n) {
        float4* dst = reinterpret_cast<float4*>(xg + (size_t)row * R + c0);
#pragma unroll
        for (int c4 = 0; c4 < kHalf / 4; ++c4) dst[c4] = make_float4(y[4 * c4], y[4 * c4 + 1], y[4 * c4 + 2], y[4 * c4 + 3]);
      }
      // the window chunks 2 g, 2 g + 1 (the last group's y is read by no MMA)
      if (g < ng - 1) put_operand(pA + LY::kWin + ((2 * g) % kNWC) * LY::kWinChunk, y, sinv);
      fence_proxy_async_smem();
      tc_fence_before();
      simt_sync();
      if (st == 0) mbar_arrive(bready);
    }
    // backward operand scale: power of two at or above max |y~| per column (rows: lanes and the four
    // quadrant warps of this column half)
    if (ok) {
#pragma unroll
      for (int c = 0; c < kHalf; ++c) {
        float m = cmax[c];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        cmax[c] = m;
      }
      if (lane == 0)
#pragma unroll
        for (int c = 0; c < kHalf; ++c) scr[(warp - 3) * kHalf + c] = cmax[c];
      simt_sync();
      if (st < R) {
        const int hh = st / kHalf, c = st % kHalf;
        float m = 0.f;
        for (int w = 0; w < 4; ++w) m = fmaxf(m, scr[(4 * hh + w) * kHalf + c]);
        sigb[st] = pow2_at_or_above(m);
      }
      simt_sync();
#pragma unroll
      for (int c = 0; c < kHalf; ++c) {
        sg[c] = sigb[c0 + c];
        sinv[c] = 1.f / sg[c];
      }
    }
    // backward
    if (ok) load_rows(ng - 1, rv);
    for (int k = 0; k < ng && ok; ++k) {
      const int g = ng - 1 - k;
      float t[kHalf];
      if (g + 1 <= ng - 1) {
        if (!(ok = decide(baccready, (uint32_t)((k - 1) & 1)))) break;
        tc_fence_after();
        tmem_pair((uint32_t)((g % 3) * 2 * kSet), t);
#pragma unroll
        for (int c = 0; c < kHalf; ++c) t[c] = rv[c] - sg[c] * t[c];
      } else {
#pragma unroll
        for (int c = 0; c < kHalf; ++c) t[c] = rv[c];
      }
      put_operand(b2p, t, sinv);
      fence_proxy_async_smem();
      tc_fence_before();
      simt_sync();
      if (st == 0) mbar_arrive(tready);
      const int row = g * kG + rq;
      const float drow = row < n ? dval(row) : 0.f;
      load_rows(g - 1, rv);
      if (!(ok = decide(yready, (uint32_t)((ng + k) & 1)))) break;
      tc_fence_after();
      float x[kHalf];
      tmem_pair(12 * R, x);
#pragma unroll
      for (int c = 0; c < kHalf; ++c) x[c] *= sg[c];
      if (row < n) {
        float4* dst = reinterpret_cast<float4*>(xg + (size_t)row * R + c0);
#pragma unroll
        for (int c4 = 0; c4 < kHalf / 4; ++c4)
          dst[c4] = make_float4(x[4 * c4] * drow, x[4 * c4 + 1] * drow, x[4 * c4 + 2] * drow, x[4 * c4 + 3] * drow);
      }
      // the MMAs of the previous group must be done with the x~ operand before it is rewritten
      if (k >= 1 && !(ok = decide(xfree, (uint32_t)((k - 1) & 1)))) break;
      put_operand(pA + LY::kWin, x, sinv);
      fence_proxy_async_smem();
      tc_fence_before();
      simt_sync();
      if (st == 0) mbar_arrive(xready);
    }
    if (!ok && st == 0) flags[0] = 1;
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(done, 0, kDrainPolls) && !flags[0];
  if (!ok && tid == 0) atomicExch(a.status, kStatusTimeout);
  if (ok) {
    // w_out[e] = 2 x_c - w_in[e], one port per thread, 16-byte rows
    for (int q = tid; q < pd.nports; q += kWtThreads) {
      const int port = pd.port_off + q;
      const float4* xr = reinterpret_cast<const float4*>(xg + (size_t)a.port_local[port] * R);
      float4 x[R / 4];
#pragma unroll
      for (int k4 = 0; k4 < R / 4; ++k4) x[k4] = xr[k4];
      for (int e = a.port_end_ptr[port]; e < a.port_end_ptr[port + 1]; ++e) {
        const float4* wi = reinterpret_cast<const float4*>(a.wprev + (size_t)a.twin[e] * R);
        float4* wo = reinterpret_cast<float4*>(a.wnext + (size_t)e * R);
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          const float4 w = wi[k4];
          wo[k4] = make_float4(2.f * x[k4].x - w.x, 2.f * x[k4].y - w.y, 2.f * x[k4].z - w.z, 2.f * x[k4].w - w.w);
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

cudaError_t wide_tc_configure(int R) {
  cudaError_t e = cudaFuncSetAttribute(k_wide_tc_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFactorSmem);
  if (e != cudaSuccess) return e;
  if (R == 16)
    return cudaFuncSetAttribute(k_sweep_wide_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WtLayout<16>::kBytes);
  if (R == 32)
    return cudaFuncSetAttribute(k_sweep_wide_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WtLayout<32>::kBytes);
  return cudaErrorInvalidValue;
}

cudaError_t launch_wide_tc_factor(const PieceDesc* pieces, int npieces, int max_groups, const float* band,
                                  unsigned char* wt, cudaStream_t st) {
  if (npieces <= 0 || max_groups <= 0) return cudaSuccess;
  k_wide_tc_factor<<<dim3(npieces, max_groups), 256, kFactorSmem, st>>>(pieces, band, wt);
  return cudaGetLastError();
}

cudaError_t launch_sweep_wide_tc(const SweepArgs<float, float>& a, int R, int npieces, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  if (!a.wt) return cudaErrorInvalidValue;
  if (R == 16) k_sweep_wide_tc<16><<<npieces, kWtThreads, WtLayout<16>::kBytes, st>>>(a);
  else if (R == 32) k_sweep_wide_tc<32><<<npieces, kWtThreads, WtLayout<32>::kBytes, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace vtm
