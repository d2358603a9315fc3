// Port-response sweep for 16 or 32 right-hand sides on the 5th-generation tensor cores.
//
// Per subgraph the sweep needs y = S_j s (then u = u_base + y, w_out = 2u - w_in; see port.cu for
// the method).  With R = 16/32 columns this is a dense product, run as tcgen05.mma (kind::f16,
// FP32 accumulation in tensor memory).
//
// Storage of S_j.  S_j is symmetric (the open-circuit impedance matrix of Def. 7.1 over all ports,
// the S of eq. A3.3), so only its lower block triangle is kept: 128 x 128 blocks (I, J), J <= I,
// row by row.  Block (I, J) serves two products: y_I += S_IJ s_J reads it K-major and
// y_J += S_IJ^T s_I reads the same bytes as an MN-major (transposed) operand.  Each block is four
// 128-byte-swizzled panels [hi, cols 0-63][hi, cols 64-127][lo, 0-63][lo, 64-127] of h_I rows
// (rows of 128 bytes, 16-byte units XOR-ed with the row mod 8, 8-row groups 1024 bytes apart);
// h_I = 128 except for the last super-row, whose height is its port count rounded up to 16.  The
// values are those of the diagonally balanced S'_j = G^-1 S_j G^-1 (G = diag(sqrt(S_pp)), so that
// S'_pp = 1 and |S'_pq| <= 1 even across coefficient jumps of many decades) divided by sigma_j, the
// power of two at or above max |S'_j|; hi = fp16(x) and lo = fp16(x - hi), so hi + lo keeps about
// 22 significant bits.  The port vector is balanced the other way (s' = G s) and y = G^-1 S' s'.  Transposed fp16 operands work on
// this tensor core; kind::tf32 with the same MN-major descriptor returns zeros, which is why the
// storage is fp16 pairs and not FP32.
//
// Products.  The port vector s = sum_e w_in[e] / Z_e (plus coupling currents) is split the same
// way per subgraph and column: s / sigma_r = s_hi + s_lo (sigma_r a power of two).  Per block and
// K step: hi(S) s_hi + hi(S) s_lo (+ lo(S) s_hi when the lo half is used), FP32 accumulation.
// With the lo half the products keep about 2^-21 of |S||s| (the dropped lo(S) s_lo term and the
// fp16 roundings); without it (FP16 storage, half the bytes) S carries fp16 rounding, 2^-11 of
// sigma_j, and the FP64 defect correction absorbs it as for the FP16 tiles of port.cu.
//
// One persistent kernel per sweep, one CTA per SM looping over subgraphs, 448 threads:
//  * warp 0 streams the blocks (and the s_J tile of off-diagonal blocks) through a ring of 16 KB
//    shared-memory slots by bulk copies (mbarrier complete_tx).  A block's panels go out one pair
//    at a time, each as soon as its slots are free, so that the next blocks stream in while the
//    current one is multiplied; the s_I tile of each super-row goes into a 2-slot row buffer a few
//    blocks before its row starts;
//  * warp 1 issues the MMAs: y_I at tensor-memory columns I R .. I R + R - 1, lane = port, all
//    super-rows of a subgraph held at once (n4 R <= 512 columns); tcgen05.commit releases stages
//    and row buffers and hands each finished y_I to the epilogue;
//  * warps 2-5 run the epilogue of the current subgraph: tcgen05.ld of each y_I (released at once
//    for the next subgraph's MMAs), u = u_base + sigma_j sigma_r y, w_out[e] = 2u - w_in[e];
//  * warps 6-13 compute the next subgraph's s: a gather pass driven by per-port records (FP32
//    values to a staging area), a coalesced pass over that area for the column maxima, then the
//    split values written to a per-CTA global scratch slot that stays in L2.
// Every wait is bounded; a CTA that gives up records VTM_ERR_TIMEOUT, lets its copies and MMAs
// finish, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include "kernels.h"
#include "tc.cuh"

namespace vtm {

using namespace tc;

namespace {

constexpr int kSB = 128;                // ports per super-block (MMA M; K extent of a block)
constexpr int kEpiWarps = 4;            // epilogue: one warp per tensor-memory lane quadrant
constexpr int kVecWarps = 8;            // port vectors
constexpr int kTcThreads = 32 * (2 + kEpiWarps + kVecWarps);  // warp 0 copies, warp 1 MMA
constexpr int kVecThreads = 32 * kVecWarps;
constexpr int kVecBar = 1;              // named barrier of the vector warps
constexpr int kEpiBar = 2;              // named barrier of the epilogue warps
constexpr int kMaxSuper = kTcMaxSuper;  // super-rows per subgraph (and tensor memory: n4 R <= 512)

__host__ __device__ __forceinline__ int n_super(int nports) { return (nports + kSB - 1) / kSB; }

// Stored rows of super-row I (a multiple of 16).
__host__ __device__ __forceinline__ int sb_rows(int nports, int I) {
  const int n4 = n_super(nports);
  if (I < n4 - 1) return kSB;
  return ((nports - kSB * I) + 15) & ~15;
}

// Byte offset of block (I, J) from the subgraph's first block (hi + lo: 512 bytes per row).
__host__ __device__ __forceinline__ int64_t blk_off(int nports, int I, int J) {
  return (int64_t)I * (I + 1) / 2 * (kSB * 512) + (int64_t)J * sb_rows(nports, I) * 512;
}

__device__ __forceinline__ void vec_sync() { asm volatile("bar.sync %0, %1;" ::"n"(kVecBar), "n"(kVecThreads) : "memory"); }
__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(kEpiBar), "n"(32 * kEpiWarps) : "memory");
}

// Header offsets (bytes from the aligned start).
constexpr uint32_t kOffFull = 0, kOffEmpty = 64, kOffRowFull = 128, kOffRowEmpty = 144, kOffSReady = 160,
                   kOffSlotFree = 176, kOffRReady = 192, kOffRowRead = 320, kOffDone = 448, kOffTslot = 456,
                   kOffFlags = 464, kOffSsig = 512, kOffOwner = 768, kOffRed = 1024;
static_assert(kOffRReady + 8 * kMaxSuper <= kOffRowRead && kOffRowRead + 8 * kMaxSuper <= kOffDone, "header");

// Shared-memory plan.  The kernel has no static shared memory: up to 1008 bytes to align the start
// to 1024, a 2 KB header (mbarriers, flags, the column scales sigma_r, the copy warp's slot owners,
// the vector warps' reduction scratch), a ring of 10 slots of 16 KB that carries the S panels and
// s_J tiles, then two s_I row tiles.  Ten slots hold two stages of an off-diagonal block with its
// lo half (four panels and the s_J tile) at once; every further slot is taken from the L1 cache that
// the gathers of the vector and epilogue warps hit in, which costs more than the extra bytes in
// flight gain (measured: 9, 10, 11, 12 slots run one sweep in 1.12, 1, 1.08, 1.10 times the time).
template <int R>
struct Plan {
  static constexpr uint32_t kSlot = 16384;              // one panel of a full-height block
  static constexpr uint32_t kVec = (uint32_t)R * 512u;  // s tile: hi / lo x 2 panels of R rows
  static constexpr uint32_t kHead = 2048;
  static constexpr int kSlots = 10;
  static constexpr uint32_t kRow = kHead + kSlots * kSlot;  // the two row tiles, from the aligned start
  static constexpr uint32_t kAlloc = 1008 + kRow + 2 * kVec;
  static_assert(kAlloc <= 227 * 1024, "shared-memory plan");
  static_assert(kOffSsig + 8 * R <= kOffOwner && kOffOwner + 4 * kSlots <= kOffRed, "header");
};
constexpr int kStg = 8;  // stage barriers (full / empty) in use round robin

// Ring slots of one block (stage).  The hi panels (and, with the lo half, the lo panels) take two
// adjacent slots each: the transposed product reads a pair as one MN-major operand whose halves are
// one slot apart, so a pair never wraps around the end of the ring.  The s_J tile of an off-diagonal
// block takes one slot, the ring's last one when a pair would otherwise start there (else that slot
// is skipped).  Copy warp and MMA issuer place the same sequence of blocks and so agree on every
// position; `a` counts slots from the start of the launch.
struct StagePos {
  int hi, lo, s;
};
template <int NS>
__device__ __forceinline__ StagePos place_stage(int64_t& a, bool lo, bool has_s) {
  StagePos p{-1, -1, -1};
  bool s_open = has_s;
  auto pair = [&]() {
    if ((int)(a % NS) == NS - 1) {
      if (s_open) {
        p.s = NS - 1;
        s_open = false;
      }
      ++a;
    }
    const int r = (int)(a % NS);
    a += 2;
    return r;
  };
  p.hi = pair();
  if (lo) p.lo = pair();
  if (s_open) {
    p.s = (int)(a % NS);
    ++a;
  }
  return p;
}

// The MMAs of one block (I, J) of height h: y_I += S_IJ s_J (A K-major: the block's two panels
// along K; B = the s tile bv) and, off the diagonal, y_J += S_IJ^T s_I (A MN-major: M over the two
// panels of a pair, one ring slot apart; K = the block's rows in steps of 16; B = the row tile si).
// Products per K step: hi(S) s_hi, hi(S) s_lo and, with LO, lo(S) s_hi.  first / first_t: the
// product overwrites y_I / y_J instead of adding.  Descriptors are formed once and advanced by
// address offsets (16-byte units in the low bits).
template <int R, bool LO>
__device__ __forceinline__ void block_mmas(uint32_t hiA, uint32_t loA, uint32_t bv, uint32_t si, int h, uint32_t dI,
                                           uint32_t dJ, bool first, bool first_t, bool transposed) {
  constexpr uint32_t idK = idesc_f16(false, R), idT = idesc_f16(true, R);
  constexpr uint32_t vpan = (uint32_t)R * 128 / 16;  // s tile panel, 16-byte units
  constexpr uint32_t pan = Plan<R>::kSlot / 16;      // ring slot, 16-byte units
  const uint64_t aK = sdesc(hiA, 16, 1024), aKl = sdesc(loA, 16, 1024);
  const uint64_t bB = sdesc(bv, 16, 1024), bR = sdesc(si, 16, 1024);
#pragma unroll
  for (int kk = 0; kk < kSB / 16; ++kk) {
    const uint32_t p = kk >> 2, o = (kk & 3) * 2;  // panel, 32-byte step in 16-byte units
    const uint64_t aH = aK + p * pan + o, bH = bB + p * vpan + o, bL = bB + (2 + p) * vpan + o;
    if (kk == 0) mma_f16(dI, aH, bH, idK, first ? 0u : 1u);
    else mma_f16_acc(dI, aH, bH, idK);
    mma_f16_acc(dI, aH, bL, idK);
    if constexpr (LO) mma_f16_acc(dI, aKl + p * pan + o, bH, idK);
  }
  if (!transposed) return;
  const uint64_t aT = sdesc(hiA, Plan<R>::kSlot, 1024), aTl = sdesc(loA, Plan<R>::kSlot, 1024);
  const int nk = h / 16;
#pragma unroll
  for (int kk = 0; kk < kSB / 16; ++kk) {
    if (kk >= nk) break;
    const uint32_t p = kk >> 2, o = (kk & 3) * 2;
    const uint64_t aH = aT + kk * 128, bH = bR + p * vpan + o, bL = bR + (2 + p) * vpan + o;  // 2048 B per kk
    if (kk == 0) mma_f16(dJ, aH, bH, idT, first_t ? 0u : 1u);
    else mma_f16_acc(dJ, aH, bH, idT);
    mma_f16_acc(dJ, aH, bL, idT);
    if constexpr (LO) mma_f16_acc(dJ, aTl + kk * 128, bH, idT);
  }
}

// s_p for one port and all R columns: sum over its ends of w_in / Z_e plus the coupling currents.
// The loads wait on a busy HBM, so they come in few dependent steps: the port's gather record
// (loaded one port ahead by the caller) gives the wave rows and coefficients of its first four
// entries, whose rows are read two at a time; entries past the fourth (rare) follow the per-port
// lists.  The additions keep the order ends-then-coupling.
template <int R>
__device__ __forceinline__ void port_vector(const PortTCArgs& a, const int4 (&rec)[3], float (&v)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = 0.f;
  const int row[4] = {rec[0].x, rec[0].y, rec[0].z, rec[0].w};
  const float c[4] = {__int_as_float(rec[1].x), __int_as_float(rec[1].y), __int_as_float(rec[1].z),
                      __int_as_float(rec[1].w)};
#pragma unroll
  for (int j = 0; j < 4; j += 2) {
    if (row[j] < 0) break;  // entries are packed, absent ones at the end
    const bool two = row[j + 1] >= 0;
    const float4* w0 = reinterpret_cast<const float4*>(a.wprev + (size_t)row[j] * R);
    const float4* w1 = reinterpret_cast<const float4*>(a.wprev + (size_t)(two ? row[j + 1] : row[j]) * R);
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const float4 x = w0[q], y = w1[q];
      v[4 * q] += x.x * c[j];
      v[4 * q + 1] += x.y * c[j];
      v[4 * q + 2] += x.z * c[j];
      v[4 * q + 3] += x.w * c[j];
      if (two) {
        v[4 * q] += y.x * c[j + 1];
        v[4 * q + 1] += y.y * c[j + 1];
        v[4 * q + 2] += y.z * c[j + 1];
        v[4 * q + 3] += y.w * c[j + 1];
      }
    }
  }
  for (int e = rec[2].x; e < rec[2].y; ++e) {
    const float4* w = reinterpret_cast<const float4*>(a.wprev + (size_t)a.twin[e] * R);
    const float iz = a.invz[e];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const float4 x = w[q];
      v[4 * q] += x.x * iz;
      v[4 * q + 1] += x.y * iz;
      v[4 * q + 2] += x.z * iz;
      v[4 * q + 3] += x.w * iz;
    }
  }
  for (int k = rec[2].z; k < rec[2].w; ++k) {
    const float yk = a.cpl.y[k];
    const float4* w = reinterpret_cast<const float4*>(a.wprev + (size_t)a.cpl.oth[k] * R);
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      const float4 x = w[q];
      v[4 * q] += yk * x.x;
      v[4 * q + 1] += yk * x.y;
      v[4 * q + 2] += yk * x.z;
      v[4 * q + 3] += yk * x.w;
    }
  }
}

}  // namespace

int64_t port_f16_bytes(int nports) {
  if (nports <= 0) return 0;
  const int n4 = n_super(nports);
  const int64_t b = blk_off(nports, n4 - 1, 0) + (int64_t)n4 * sb_rows(nports, n4 - 1) * 512;
  return (b + 1023) & ~int64_t(1023);
}

int64_t port_f32_blocks(int nports) {
  const int64_t n4 = n_super(nports);
  return n4 * (n4 + 1) / 2;
}

size_t port_tc_smem_bytes(int R, bool) { return R == 16 ? Plan<16>::kAlloc : Plan<32>::kAlloc; }

// S_j columns cc = b * Rs + r from unit-source solves into FP32 128 x 128 row-major blocks of the
// lower block triangle (block (I, J) at s_off + I (I + 1) / 2 + J; diagonal blocks whole).
__global__ void k_gather_port_blocks(const PieceDesc* __restrict__ pieces, const int32_t* __restrict__ port_local,
                                     int Rs, int b, const float* __restrict__ xc, float* __restrict__ S32) {
  const PieceDesc pd = pieces[blockIdx.x];
  for (int i = threadIdx.x; i < pd.nports * Rs; i += blockDim.x) {
    const int q = i / Rs, r = i % Rs;
    const int cc = b * Rs + r;
    if (cc >= pd.nports) continue;
    const int I = q / kSB, J = cc / kSB;
    if (J > I) continue;
    const int64_t blk = pd.s_off + (int64_t)I * (I + 1) / 2 + J;
    S32[blk * (kSB * kSB) + (q % kSB) * kSB + cc % kSB] =
        xc[((size_t)pd.copy_off + port_local[pd.port_off + q]) * Rs + r];
  }
}

// FP32 blocks -> fp16 hi / lo panels of the sweep's layout.  S_j is first balanced by its diagonal,
// S'_pq = S_pq / (g_p g_q) with g_p = sqrt(S_pp) (so S'_pp = 1 and |S'_pq| <= 1, S_j being SPD):
// across a coefficient jump the entries of S_j span many decades (a soft region's input impedances
// are orders of magnitude above a stiff one's), which one scale per subgraph would push below the
// fp16 range.  g_p goes to gscale[port]; sigma_j = 2^e >= max |S'| (about 1) to sig.
__global__ void k_port_blocks_to_f16(const PieceDesc* __restrict__ pieces, const float* __restrict__ S32,
                                     unsigned char* __restrict__ S16, float* __restrict__ sig,
                                     float* __restrict__ gscale) {
  const PieceDesc pd = pieces[blockIdx.x];
  const int P = pd.nports;
  if (P == 0) return;
  const int n4 = n_super(P);
  const float* src = S32 + pd.s_off * (kSB * kSB);
  __shared__ float g[kMaxSuper * kSB];  // 1 / g_p, zero-padded
  __shared__ float red[32];
  for (int p = threadIdx.x; p < n4 * kSB; p += blockDim.x) {
    float gi = 0.f;
    if (p < P) {
      const int I = p / kSB, r = p % kSB;
      const float d = src[((int64_t)I * (I + 1) / 2 + I) * (kSB * kSB) + r * kSB + r];
      const float gp = d > 0.f ? sqrtf(d) : 1.f;
      gscale[pd.port_off + p] = gp;
      gi = 1.f / gp;
    }
    g[p] = gi;
  }
  __syncthreads();
  float m = 0.f;
  for (int I = 0; I < n4; ++I)
    for (int J = 0; J <= I; ++J) {
      const float* blk = src + ((int64_t)I * (I + 1) / 2 + J) * (kSB * kSB);
      for (int k = threadIdx.x; k < kSB * kSB; k += blockDim.x)
        m = fmaxf(m, fabsf(blk[k] * g[I * kSB + k / kSB] * g[J * kSB + k % kSB]));
    }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
    int e = 0;
    if (mm > 0.f) frexpf(mm, &e);
    red[0] = ldexpf(1.f, e);  // power of two >= mm (1 for an all-zero matrix)
    sig[blockIdx.x] = red[0];
  }
  __syncthreads();
  const float inv = 1.f / red[0];
  unsigned char* dst = S16 + pd.h_off;
  for (int I = 0; I < n4; ++I) {
    const int h = sb_rows(P, I);
    for (int J = 0; J <= I; ++J) {
      const float* blk = src + ((int64_t)I * (I + 1) / 2 + J) * (kSB * kSB);
      unsigned char* o = dst + blk_off(P, I, J);
      const uint32_t panel = (uint32_t)h * 128;
      for (int k = threadIdx.x; k < h * kSB; k += blockDim.x) {
        const int row = k / kSB, col = k % kSB;
        const float x = blk[k] * g[I * kSB + row] * g[J * kSB + col] * inv;
        const __half hi = __float2half_rn(x);
        const __half lo = __float2half_rn(x - __half2float(hi));
        const uint32_t off = (uint32_t)(col / 64) * panel + swz16(row, col % 64);
        *reinterpret_cast<__half*>(o + off) = hi;
        *reinterpret_cast<__half*>(o + 2 * panel + off) = lo;
      }
    }
  }
}

template <int R, bool LO>
__global__ void __launch_bounds__(kTcThreads, 1) k_port_sweep_tc(const PortTCArgs a) {
  using P = Plan<R>;
  constexpr int NS = P::kSlots;
  static_assert(kVecThreads % (R / 4) == 0 && 32 % (R / 4) == 0, "column groups of the maxima pass");
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kOffFull);          // [kStg] stage landed
  uint64_t* empty = reinterpret_cast<uint64_t*>(sm + kOffEmpty);        // [kStg] MMAs done with the stage
  uint64_t* rowfull = reinterpret_cast<uint64_t*>(sm + kOffRowFull);    // [2] s_I tile landed
  uint64_t* rowempty = reinterpret_cast<uint64_t*>(sm + kOffRowEmpty);  // [2] MMAs done with the s_I tile
  uint64_t* sready = reinterpret_cast<uint64_t*>(sm + kOffSReady);      // [2] scratch slot written
  uint64_t* slotfree = reinterpret_cast<uint64_t*>(sm + kOffSlotFree);  // [2] epilogue of the slot's last subgraph done
  uint64_t* rready = reinterpret_cast<uint64_t*>(sm + kOffRReady);      // [kMaxSuper] accumulator y_I complete
  uint64_t* rowread = reinterpret_cast<uint64_t*>(sm + kOffRowRead);    // [kMaxSuper] y_I read by the epilogue
  uint64_t* done = reinterpret_cast<uint64_t*>(sm + kOffDone);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffTslot);
  volatile int* flags = reinterpret_cast<volatile int*>(sm + kOffFlags);  // abort, epilogue stop, vector stop
  float (*ssig)[R] = reinterpret_cast<float (*)[R]>(sm + kOffSsig);        // [2][R] sigma_r per scratch slot
  float (*red)[R] = reinterpret_cast<float (*)[R]>(sm + kOffRed);          // [kVecWarps][R]
  const uint32_t ring = base + P::kHead;
  const uint32_t row0 = base + P::kRow;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npc = (a.npieces - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // subgraphs of this CTA
  const size_t slot_bytes = (size_t)a.n4max * P::kVec;
  unsigned char* scratch = a.scratch + (size_t)blockIdx.x * (2 * slot_bytes + (size_t)a.n4max * kSB * R * 4);
  float* stage32 = reinterpret_cast<float*>(scratch + 2 * slot_bytes);  // FP32 port vectors, ports x R

  if (tid == 0) {
    flags[0] = flags[1] = flags[2] = 0;
    for (int s = 0; s < kStg; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&rowfull[s], 1);
      mbar_init(&rowempty[s], 1);
      mbar_init(&sready[s], 1);
      mbar_init(&slotfree[s], 1);
    }
    for (int s = 0; s < kMaxSuper; ++s) {
      mbar_init(&rready[s], 1);
      mbar_init(&rowread[s], kEpiWarps);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  volatile int& abort_flag = flags[0];

  if (warp == 0) {
    // ---- copies: super-rows in descending order; per block (I, J), J = I .. 0, its panels and
    // (off the diagonal) the s_J tile; the s_I tile of the next super-row a few blocks ahead.  Each piece goes out as soon as
    // its slots are free (the MMAs of the stage that last filled them are complete), so the next
    // blocks stream in while the current one is multiplied; the stage's full barrier counts the
    // bytes of every piece and completes after the last piece has been issued and has landed.
    // The blocks are read once per sweep: evict first.
    if (lane == 0) {
      uint64_t policy;
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
      // stage that last filled each slot, in shared memory: a local array would sit in a cache that
      // the ring leaves small, and this one thread issues every copy
      int* owner = reinterpret_cast<int*>(sm + kOffOwner);
      for (int i = 0; i < NS; ++i) owner[i] = -1;
      int gblk = 0, rel = -1;  // rel: stages 0 .. rel known released
      int64_t grow = 0, aslot = 0;
      auto release_upto = [&](int j) -> bool {
        while (rel < j) {
          ++rel;
          if (!mbar_wait_bounded(&empty[rel % kStg], (uint32_t)((rel / kStg) & 1), a.wait_limit)) return false;
        }
        return true;
      };
      for (int k = 0; k < npc && !abort_flag; ++k) {
        const PieceDesc pd = a.pieces[blockIdx.x + (size_t)k * gridDim.x];
        const int Pn = pd.nports, n4 = n_super(Pn);
        if (!mbar_wait_bounded(&sready[k & 1], (uint32_t)((k >> 1) & 1), a.wait_limit)) {
          abort_flag = 1;
          break;
        }
        const unsigned char* slot = scratch + (size_t)(k & 1) * slot_bytes;
        const unsigned char* Sp = a.S16 + pd.h_off;
        // s_I tile of super-row I into the row buffer grow & 1, once the MMAs of the row two
        // before it (same buffer) are done
        auto issue_row = [&](int I) -> bool {
          const int rb = (int)(grow & 1);
          if (grow >= 2 && !mbar_wait_bounded(&rowempty[rb], (uint32_t)(((grow >> 1) - 1) & 1), a.wait_limit))
            return false;
          mbar_arrive_expect_tx(&rowfull[rb], P::kVec);
          bulk_g2s(row0 + rb * P::kVec, slot + (size_t)I * P::kVec, P::kVec, &rowfull[rb]);
          ++grow;
          return true;
        };
        if (n4 > 0 && !issue_row(n4 - 1)) {
          abort_flag = 1;
          break;
        }
        for (int I = n4 - 1; I >= 0 && !abort_flag; --I) {
          const int h = sb_rows(Pn, I);
          const uint32_t pbytes = (uint32_t)h * 128;  // one panel
          for (int J = I; J >= 0; --J) {
            const int st = (int)(gblk % kStg);
            // full[st] and empty[st] were last used by stage gblk - kStg
            bool ok = release_upto(gblk - kStg);
            const StagePos ps = place_stage<NS>(aslot, LO, J < I);
            const unsigned char* blk = Sp + blk_off(Pn, I, J);
            // one pair: two panels of the block into two adjacent slots
            auto pair = [&](int s0, const unsigned char* src) {
              ok = ok && release_upto(owner[s0] > owner[s0 + 1] ? owner[s0] : owner[s0 + 1]);
              if (!ok) return;
              owner[s0] = owner[s0 + 1] = gblk;
              const uint32_t dst = ring + (uint32_t)s0 * P::kSlot;
              mbar_expect_tx(&full[st], 2 * pbytes);
              if (h == kSB) {
                bulk_g2s_hint(dst, src, 2 * pbytes, &full[st], policy);
              } else {
                bulk_g2s_hint(dst, src, pbytes, &full[st], policy);
                bulk_g2s_hint(dst + P::kSlot, src + pbytes, pbytes, &full[st], policy);
              }
            };
            pair(ps.hi, blk);
            if (LO) pair(ps.lo, blk + 2 * pbytes);
            if (ps.s >= 0) {
              ok = ok && release_upto(owner[ps.s]);
              if (ok) {
                owner[ps.s] = gblk;
                mbar_expect_tx(&full[st], P::kVec);
                bulk_g2s(ring + (uint32_t)ps.s * P::kSlot, slot + (size_t)J * P::kVec, P::kVec, &full[st]);
              }
            }
            mbar_arrive(&full[st]);  // completes once what was issued has landed
            ++gblk;
            // the next row's tile goes out a few blocks ahead: by the third block of this row the
            // MMAs have finished the row before it, whose buffer it takes
            if (ok && I > 0 && J == (I >= 2 ? I - 2 : 0)) ok = issue_row(I - 1);
            if (!ok) {
              abort_flag = 1;
              break;
            }
          }
        }
      }
      // copies still in flight must land before the shared memory can go away
      for (int g = (gblk > kStg ? gblk - kStg : 0); g < gblk; ++g)
        mbar_wait_bounded(&full[g % kStg], (uint32_t)((g / kStg) & 1), kDrainPolls);
      for (int64_t g = (grow > 2 ? grow - 2 : 0); g < grow; ++g)
        mbar_wait_bounded(&rowfull[g & 1], (uint32_t)((g >> 1) & 1), kDrainPolls);
    }
  } else if (warp == 1) {
    // ---- MMA issuer.  In descending row order y_I is complete once row I is done (the rows
    // below only add to y_J, J < I), so its epilogue runs while the MMAs go on.  The first row
    // processed (n4 - 1) initialises every accumulator: y_{n4-1} through the direct product of the
    // diagonal block, every other y_J through the transposed product of block (n4 - 1, J).  Before
    // it overwrites y_J it waits until the epilogue has read y_J of the subgraph before (rowread);
    // that subgraph's epilogue reads its rows in the same descending order, so the MMAs of the
    // next subgraph start while the last rows of this one are still being written out.
    if (lane == 0) {
      int64_t gblk = 0, grow = 0, aslot = 0;
      uint32_t pend = 0, wpar = 0;  // rows handed to the epilogue and not yet waited for; parity of the next wait
      for (int k = 0; k < npc && !abort_flag; ++k) {
        const PieceDesc pd = a.pieces[blockIdx.x + (size_t)k * gridDim.x];
        const int Pn = pd.nports, n4 = n_super(Pn);
        for (int I = n4 - 1; I >= 0 && !abort_flag; --I) {
          const int rb = (int)(grow & 1);
          if (!mbar_wait_bounded(&rowfull[rb], (uint32_t)((grow >> 1) & 1), a.wait_limit)) {
            abort_flag = 1;
            break;
          }
          const uint32_t si = row0 + rb * P::kVec;
          const int h = sb_rows(Pn, I);
          const bool top = (I == n4 - 1);
          for (int J = I; J >= 0; --J) {
            const int st = (int)(gblk % kStg);
            const StagePos ps = place_stage<NS>(aslot, LO, J < I);
            if (top && ((pend >> J) & 1u)) {  // first write into y_J (y_I on the diagonal) this subgraph
              if (!mbar_wait_bounded(&rowread[J], (wpar >> J) & 1u, a.wait_limit)) {
                abort_flag = 1;
                break;
              }
              wpar ^= 1u << J;
              pend &= ~(1u << J);
            }
            if (!mbar_wait_bounded(&full[st], (uint32_t)((gblk / kStg) & 1), a.wait_limit)) {
              abort_flag = 1;
              break;
            }
            tc_fence_after();
            const uint32_t hiA = ring + (uint32_t)ps.hi * P::kSlot;
            const uint32_t loA = LO ? ring + (uint32_t)ps.lo * P::kSlot : hiA;
            const uint32_t bv = (J == I) ? si : ring + (uint32_t)ps.s * P::kSlot;
            const uint32_t dI = tmem + (uint32_t)(I * R), dJ = tmem + (uint32_t)(J * R);
            block_mmas<R, LO>(hiA, loA, bv, si, h, dI, dJ, top && J == I, top, J < I);
            mma_commit(&empty[st]);
            ++gblk;
          }
          mma_commit(&rowempty[rb]);
          mma_commit(&rready[I]);  // y_I is final
          ++grow;
        }
        pend |= (n4 >= 32 ? ~0u : (1u << n4) - 1u);
      }
      mma_commit(done);  // arrives once every MMA issued above has completed
    }
  } else if (warp < 2 + kEpiWarps) {
    // ---- epilogue warps (one per tensor-memory lane quadrant): u = u_base + sigma_j sigma_r y_I,
    // w_out[e] = 2 u - w_in[e], super-row by super-row as the MMA issuer completes them
    // (rready[I] completes once per subgraph that has a super-row I, so its phases are counted per
    // barrier; sready[k & 1] also orders the sigma_r written with subgraph k's port vectors).
    // Each warp releases y_I (rowread[I]) as soon as its tcgen05.ld has completed.
    const int q = warp & 3;
    uint32_t uses = 0;  // tid 64: parity of the next phase of each row barrier, one bit per super-row
    bool stop = false;
    for (int k = 0; k < npc && !stop; ++k) {
      const PieceDesc pd = a.pieces[blockIdx.x + (size_t)k * gridDim.x];
      const int Pn = pd.nports, n4 = n_super(Pn);
      const float sj = a.sig_s[blockIdx.x + (size_t)k * gridDim.x];
      if (tid == 64) flags[1] = mbar_wait_bounded(&sready[k & 1], (uint32_t)((k >> 1) & 1), a.wait_limit) ? 0 : 1;
      epi_sync();
      stop = flags[1] != 0;
      epi_sync();
      for (int I = n4 - 1; I >= 0 && !stop; --I) {
        // the four warps decide together: one lane waits, the named barrier publishes the outcome
        if (tid == 64) {
          flags[1] = mbar_wait_bounded(&rready[I], (uses >> I) & 1u, a.wait_limit) ? 0 : 1;
          uses ^= 1u << I;
        }
        epi_sync();
        stop = flags[1] != 0;
        epi_sync();
        if (stop) break;
        tc_fence_after();
        uint32_t v[R];
        tmem_ld<R>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(I * R), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&rowread[I]);
        const int p = I * kSB + 32 * q + lane;
        if (p < Pn) {
          const int port = pd.port_off + p;
          const float4* ub = reinterpret_cast<const float4*>(a.ubase + (size_t)port * R);
          const int e0 = a.port_end_ptr[port], e1 = a.port_end_ptr[port + 1];
          const float gs = sj * a.gscale[port];  // y = D^-1 (sigma_j S'') (sigma_r s'')
#pragma unroll
          for (int k4 = 0; k4 < R / 4; ++k4) {
            const float4 b4 = __ldg(ub + k4);
            const float u0 = b4.x + gs * ssig[k & 1][4 * k4] * __uint_as_float(v[4 * k4]);
            const float u1 = b4.y + gs * ssig[k & 1][4 * k4 + 1] * __uint_as_float(v[4 * k4 + 1]);
            const float u2 = b4.z + gs * ssig[k & 1][4 * k4 + 2] * __uint_as_float(v[4 * k4 + 2]);
            const float u3 = b4.w + gs * ssig[k & 1][4 * k4 + 3] * __uint_as_float(v[4 * k4 + 3]);
            v[4 * k4] = __float_as_uint(u0);
            v[4 * k4 + 1] = __float_as_uint(u1);
            v[4 * k4 + 2] = __float_as_uint(u2);
            v[4 * k4 + 3] = __float_as_uint(u3);
          }
          for (int e = e0; e < e1; ++e) {
            const float4* wi = reinterpret_cast<const float4*>(a.wprev + (size_t)a.twin[e] * R);
            float4* wo = reinterpret_cast<float4*>(a.wnext + (size_t)e * R);
#pragma unroll
            for (int k4 = 0; k4 < R / 4; ++k4) {
              const float4 w = __ldg(wi + k4);
              wo[k4] = make_float4(2.f * __uint_as_float(v[4 * k4]) - w.x, 2.f * __uint_as_float(v[4 * k4 + 1]) - w.y,
                                   2.f * __uint_as_float(v[4 * k4 + 2]) - w.z,
                                   2.f * __uint_as_float(v[4 * k4 + 3]) - w.w);
            }
          }
        }
      }
      if (stop) {
        if (tid == 64) abort_flag = 1;
        break;
      }
      epi_sync();
      if (tid == 64) mbar_arrive(&slotfree[k & 1]);
    }
  } else {
    // ---- vector warps: the port vectors s of subgraph k, one gather pass (FP32 values to a
    // staging area and the column maxima), then the fp16 split into the scratch slot k & 1.  Slot
    // and sigma_r of subgraph k are free again once the epilogue of subgraph k - 2 is done
    // (slotfree[k & 1] completes once per subgraph of that slot).
    const int vt = tid - 32 * (2 + kEpiWarps);
    const int vw = vt >> 5;
    for (int k = 0; k < npc; ++k) {
      if (k >= 2) {
        if (vt == 0) flags[2] = mbar_wait_bounded(&slotfree[k & 1], (uint32_t)(((k >> 1) - 1) & 1), a.wait_limit) ? 0 : 1;
        vec_sync();
        const bool stop = flags[2] != 0;
        vec_sync();
        if (stop) {
          if (vt == 0) abort_flag = 1;
          break;
        }
      }
      const PieceDesc pd = a.pieces[blockIdx.x + (size_t)k * gridDim.x];
      const int Pn = pd.nports, np = n_super(Pn) * kSB;
      // gather: s' = D^-1 s per port into the FP32 staging area; the next port's record is
      // loaded before this port's wave rows
      int4 rec[3];
      if (vt < Pn)
#pragma unroll
        for (int i = 0; i < 3; ++i) rec[i] = a.prec[3 * (size_t)(pd.port_off + vt) + i];
      for (int p = vt; p < Pn; p += kVecThreads) {
        int4 nrec[3];
        if (p + kVecThreads < Pn)
#pragma unroll
          for (int i = 0; i < 3; ++i) nrec[i] = a.prec[3 * (size_t)(pd.port_off + p + kVecThreads) + i];
        float v[R];
        port_vector<R>(a, rec, v);
        const float gp = a.gscale[pd.port_off + p];  // s' = D^-1 s, D = diag(1 / g)
        float4* o = reinterpret_cast<float4*>(stage32 + (size_t)p * R);
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4)
          o[k4] = make_float4(v[4 * k4] * gp, v[4 * k4 + 1] * gp, v[4 * k4 + 2] * gp, v[4 * k4 + 3] * gp);
#pragma unroll
        for (int i = 0; i < 3; ++i) rec[i] = nrec[i];
      }
      vec_sync();
      // column maxima in a coalesced pass over the staged values: the thread stride is a multiple
      // of R / 4, so every float4 a thread reads holds the same four columns
      {
        float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4* s4 = reinterpret_cast<const float4*>(stage32);
        for (int i = vt; i < Pn * (R / 4); i += kVecThreads) {
          const float4 x = s4[i];
          m4 = make_float4(fmaxf(m4.x, fabsf(x.x)), fmaxf(m4.y, fabsf(x.y)), fmaxf(m4.z, fabsf(x.z)),
                           fmaxf(m4.w, fabsf(x.w)));
        }
#pragma unroll
        for (int o = R / 4; o < 32; o <<= 1) {
          m4.x = fmaxf(m4.x, __shfl_xor_sync(0xffffffffu, m4.x, o));
          m4.y = fmaxf(m4.y, __shfl_xor_sync(0xffffffffu, m4.y, o));
          m4.z = fmaxf(m4.z, __shfl_xor_sync(0xffffffffu, m4.z, o));
          m4.w = fmaxf(m4.w, __shfl_xor_sync(0xffffffffu, m4.w, o));
        }
        if (lane < R / 4) {
          red[vw][4 * lane] = m4.x;
          red[vw][4 * lane + 1] = m4.y;
          red[vw][4 * lane + 2] = m4.z;
          red[vw][4 * lane + 3] = m4.w;
        }
      }
      vec_sync();
      if (vt < R) {
        float m = 0.f;
        for (int w = 0; w < kVecWarps; ++w) m = fmaxf(m, red[w][vt]);
        int e = 0;
        if (m > 0.f) frexpf(m, &e);
        ssig[k & 1][vt] = ldexpf(1.f, e);  // power of two >= max |s_r|
      }
      vec_sync();
      unsigned char* slot = scratch + (size_t)(k & 1) * slot_bytes;
      for (int p = vt; p < np; p += kVecThreads) {
        unsigned char* tile = slot + (size_t)(p / kSB) * P::kVec;
        const int c = p % kSB;
        const uint32_t pn = (uint32_t)(c / 64) * R * 128;
        const float4* src = reinterpret_cast<const float4*>(stage32 + (size_t)p * R);
#pragma unroll
        for (int k4 = 0; k4 < R / 4; ++k4) {
          const float4 x4 = (p < Pn) ? src[k4] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = 4 * k4 + i;
            const float x = xs[i] / ssig[k & 1][r];
            const __half hi = __float2half_rn(x);
            const __half lo = __float2half_rn(x - __half2float(hi));
            const uint32_t off = pn + swz16(r, c % 64);
            *reinterpret_cast<__half*>(tile + off) = hi;
            *reinterpret_cast<__half*>(tile + 2 * R * 128 + off) = lo;
          }
        }
      }
      // the bulk copies (async proxy) read what these generic stores wrote
      asm volatile("fence.proxy.async.global;" ::: "memory");
      vec_sync();
      if (vt == 0) mbar_arrive(&sready[k & 1]);
    }
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(done, 0, kDrainPolls) && !abort_flag;
  if (!ok && tid == 0) atomicExch(a.status, kStatusTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// Gather record of port q: the wave rows and coefficients of its first four entries in the order
// the sweep adds them (ends e0 .. e1 - 1 with 1 / Z_e, then coupling entries k0 .. k1 - 1 with y;
// row -1 and coefficient 0 past the last one), and where the remaining entries resume.
__global__ void k_port_records(int nports, const int32_t* __restrict__ port_end_ptr, const int32_t* __restrict__ twin,
                               const float* __restrict__ invz, CoupleRef<float> cpl, int4* __restrict__ rec) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nports) return;
  const int e0 = port_end_ptr[q], e1 = port_end_ptr[q + 1];
  const int k0 = cpl.ptr ? cpl.ptr[q] : 0, k1 = cpl.ptr ? cpl.ptr[q + 1] : 0;
  int row[4] = {-1, -1, -1, -1};
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  int n = 0, e = e0, k = k0;
  for (; e < e1 && n < 4; ++e, ++n) {
    row[n] = twin[e];
    c[n] = invz[e];
  }
  for (; e == e1 && k < k1 && n < 4; ++k, ++n) {
    row[n] = cpl.oth[k];
    c[n] = cpl.y[k];
  }
  rec[3 * (size_t)q] = make_int4(row[0], row[1], row[2], row[3]);
  rec[3 * (size_t)q + 1] = make_int4(__float_as_int(c[0]), __float_as_int(c[1]), __float_as_int(c[2]), __float_as_int(c[3]));
  rec[3 * (size_t)q + 2] = make_int4(e, e1, k, k1);
}

cudaError_t launch_port_records(int nports, const int32_t* port_end_ptr, const int32_t* twin, const float* invz,
                                CoupleRef<float> cpl, int4* rec, cudaStream_t st) {
  if (nports <= 0) return cudaSuccess;
  k_port_records<<<(nports + 255) / 256, 256, 0, st>>>(nports, port_end_ptr, twin, invz, cpl, rec);
  return cudaGetLastError();
}

cudaError_t port_tc_configure(int R) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (R) {
    case 16:
      e = cudaFuncSetAttribute(k_port_sweep_tc<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)port_tc_smem_bytes(16, true));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_port_sweep_tc<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)port_tc_smem_bytes(16, false));
      break;
    case 32:
      e = cudaFuncSetAttribute(k_port_sweep_tc<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)port_tc_smem_bytes(32, true));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_port_sweep_tc<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)port_tc_smem_bytes(32, false));
      break;
    default: break;
  }
  return e;
}

cudaError_t launch_port_sweep_tc(const PortTCArgs& a, int R, bool lo, int grid, cudaStream_t st) {
  if (a.npieces <= 0 || grid <= 0) return cudaSuccess;
  const size_t smem = port_tc_smem_bytes(R, lo);
  if (R == 16) {
    if (lo) k_port_sweep_tc<16, true><<<grid, kTcThreads, smem, st>>>(a);
    else k_port_sweep_tc<16, false><<<grid, kTcThreads, smem, st>>>(a);
  } else if (R == 32) {
    if (lo) k_port_sweep_tc<32, true><<<grid, kTcThreads, smem, st>>>(a);
    else k_port_sweep_tc<32, false><<<grid, kTcThreads, smem, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_port_blocks(const PieceDesc* pieces, int npieces, const int32_t* port_local, int Rs, int b,
                                      const float* xc, float* S32, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_gather_port_blocks<<<npieces, 256, 0, st>>>(pieces, port_local, Rs, b, xc, S32);
  return cudaGetLastError();
}

cudaError_t launch_port_blocks_to_f16(const PieceDesc* pieces, int npieces, const float* S32, unsigned char* S16,
                                      float* sig, float* gscale, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  k_port_blocks_to_f16<<<npieces, 256, 0, st>>>(pieces, S32, S16, sig, gscale);
  return cudaGetLastError();
}

}  // namespace vtm
