// One VTM sweep over all subgraphs (Table 1 steps 3-5; eq. 5.6, 5.8), one CTA per subgraph.
//
// Per subgraph j the CTA
//   1. gathers the incident wave of each line end from its twin, w_in[e] = w_prev[twin(e)]
//      (the N2N exchange), and forms r_j = b̃_j + sum_e w_in[e]/Z_e e_c (eq. 5.8 right side);
//   2. streams the band factor of K_j from HBM in kNB-row slabs with the TMA bulk-copy engine
//      (cp.async.bulk into a ring of shared-memory stages tracked by mbarriers) and runs the
//      forward substitution L y = r on rows of L and the back substitution L^T x = y on rows of
//      U = L^T (both in dot form: 16-byte shared loads, independent FMA chains, 8-lane shuffle
//      reductions) with the diagonal blocks stored as inverses;
//   3. emits w_out[e] = 2 x_c - w_in[e] for every end (u - Z omega of eq. 5.6, written as the
//      single wave that the twin receives next sweep).
// The vector state of the subgraph (y / x: Wp-1 zero rows, n_pad rows, Wp-1 zero rows, x R) stays in
// shared memory.
#include "kernels.h"

namespace vtm {

template <typename T, typename TV, int R>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweep(const SweepArgs<T, TV> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int S = a.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  T* ring = reinterpret_cast<T*>(smem + 128);
  T* ys = ring + (size_t)S * a.slot_elems;
  T* win = ys + a.ys_elems;
  T* tb = win + a.win_elems;

  const int Wp = pd.Wp;
  const int off = Wp - 1;  // ys row of column 0
  const int nblk = pd.n_pad / kNB;
  const int total = 2 * nblk;
  const uint32_t slab_bytes = (uint32_t)(kNB * Wp * sizeof(T));
  const T* fbase = a.factor + pd.factor_off;
  const T* ubase = a.factor_u + pd.factor_off;

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
    bulk_copy_g2s(ring + (size_t)slot * a.slot_elems, (s < nblk ? fbase : ubase) + (size_t)kb * kNB * Wp, slab_bytes,
                  &bars[slot]);
  };
  if (tid == 0)
    for (int s = 0; s < S && s < total; ++s) issue(s);

  // ---- prologue: r_j = b̃_j + sum_e w_in[e] / Z_e at the port rows
  for (int i = tid; i < off * R; i += kSweepThreads) {
    ys[i] = T(0);
    ys[(size_t)(off + pd.n_pad) * R + i] = T(0);
  }
  const TV* btp = a.bt + (size_t)pd.copy_off * R;
  for (int i = tid; i < pd.n_pad * R; i += kSweepThreads) ys[(size_t)off * R + i] = (i < pd.n * R) ? (T)btp[i] : T(0);
  __syncthreads();
  for (int q = tid; q < pd.nports; q += kSweepThreads) {
    const int l = a.port_local[pd.port_off + q];
    const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
    T acc[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
    for (int e = e0; e < e1; ++e) {
      const int tw = a.twin[e];
      const T iz = (T)a.invz[e];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const T w = (T)a.wprev[(size_t)tw * R + rr];
        win[(e - pd.end_off) * R + rr] = w;
        acc[rr] += w * iz;
      }
    }
    if (a.cpl.ptr)
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] += coupling_current<T, TV>(a.cpl, pd.port_off + q, rr, R, a.wprev);
#pragma unroll
    for (int rr = 0; rr < R; ++rr) ys[(size_t)(off + l) * R + rr] += acc[rr];
  }
  __syncthreads();

  // ---- forward (s < nblk) then backward (s >= nblk) over the staged slabs
  const int rg = tid >> 3, g = tid & 7;
  int s = 0;
  for (; s < total; ++s) {
    const int slot = s % S;
    if (!mbar_wait_bounded(&bars[slot], (uint32_t)((s / S) & 1), a.wait_limit)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    const T* L = ring + (size_t)slot * a.slot_elems;
    if (s < nblk) {
      const int k0 = s * kNB;
      // t_r = r_r - sum_{col < k0} L[r][col] y_col   (positions p < off - r of row r)
      const T* Lr = L + rg * Wp;
      const int pend = off - rg;
      const T* yb = ys + (size_t)(k0 + rg) * R;
      T acc[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
      if constexpr (sizeof(T) == 4 && R == 1) {
        // 16-byte loads of the factor row; four independent FMA chains
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float4* L4 = reinterpret_cast<const float4*>(Lr);
        const int nchunk = (pend + 3) >> 2;
        for (int q = g; q < nchunk; q += 8) {
          const float4 l = L4[q];
          const int p = q << 2;
          const float* y = reinterpret_cast<const float*>(yb) + p;
          a0 = fmaf(l.x, y[0], a0);
          if (p + 1 < pend) a1 = fmaf(l.y, y[1], a1);
          if (p + 2 < pend) a2 = fmaf(l.z, y[2], a2);
          if (p + 3 < pend) a3 = fmaf(l.w, y[3], a3);
        }
        acc[0] = (a0 + a1) + (a2 + a3);
      } else {
        for (int p = g; p < pend; p += 8) {
          const T l = Lr[p];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) acc[rr] += l * yb[(size_t)p * R + rr];
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = warp_sum_g8(acc[rr]);
      if (g == 0)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) tb[rg * R + rr] = ys[(size_t)(k0 + rg + off) * R + rr] - acc[rr];
      __syncthreads();
      // y_B = inv(L_KK) t
      T acc2[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc2[rr] = T(0);
      for (int c = g; c <= rg; c += 8) {
        const T l = Lr[off - rg + c];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) acc2[rr] += l * tb[c * R + rr];
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc2[rr] = warp_sum_g8(acc2[rr]);
      if (g == 0)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) ys[(size_t)(k0 + rg + off) * R + rr] = acc2[rr];
    } else {
      const int k0 = (total - 1 - s) * kNB;
      // rows of U = L^T: t_r = y_r - sum_{col > k0+31} U[r][col] x_col  (positions p >= 32 - r)
      const T* Ur = L + rg * Wp;
      const int pbeg = kNB - rg;
      const T* xb = ys + (size_t)(k0 + rg + off) * R;
      T acc[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
      if constexpr (sizeof(T) == 4 && R == 1) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float4* U4 = reinterpret_cast<const float4*>(Ur);
        const int nchunk = Wp >> 2;
        for (int q = (pbeg >> 2) + g; q < nchunk; q += 8) {
          const float4 u = U4[q];
          const int p = q << 2;
          const float* x = reinterpret_cast<const float*>(xb) + p;
          if (p >= pbeg) a0 = fmaf(u.x, x[0], a0);
          if (p + 1 >= pbeg) a1 = fmaf(u.y, x[1], a1);
          if (p + 2 >= pbeg) a2 = fmaf(u.z, x[2], a2);
          a3 = fmaf(u.w, x[3], a3);  // p + 3 >= pbeg always holds for chunks at or after pbeg / 4
        }
        acc[0] = (a0 + a1) + (a2 + a3);
      } else {
        for (int p = pbeg + g; p < Wp; p += 8) {
          const T u = Ur[p];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) acc[rr] += u * xb[(size_t)p * R + rr];
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = warp_sum_g8(acc[rr]);
      if (g == 0)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) tb[rg * R + rr] = xb[rr] - acc[rr];
      __syncthreads();
      // x_B = inv(U_KK) t: x_r = sum_{c >= r} inv(U_KK)[r][c] t_c at positions c - r
      T acc2[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc2[rr] = T(0);
      for (int c = rg + g; c < kNB; c += 8) {
        const T u = Ur[c - rg];
#pragma unroll
        for (int rr = 0; rr < R; ++rr) acc2[rr] += u * tb[c * R + rr];
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc2[rr] = warp_sum_g8(acc2[rr]);
      if (g == 0)
#pragma unroll
        for (int rr = 0; rr < R; ++rr) ys[(size_t)(k0 + rg + off) * R + rr] = acc2[rr];
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
      // drain the copies still in flight (bounded) before the CTA leaves
      for (int s2 = s; s2 < total && s2 < s + S; ++s2)
        if (s2 != a.withhold) mbar_wait_bounded(&bars[s2 % S], (uint32_t)((s2 / S) & 1), kDrainPolls);
    }
    return;
  }

  // ---- epilogue: w_out[e] = 2 x_c - w_in[e]; local solution
  for (int q = tid; q < pd.nports; q += kSweepThreads) {
    const int l = a.port_local[pd.port_off + q];
    const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
    for (int e = e0; e < e1; ++e)
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        a.wnext[(size_t)e * R + rr] = (TV)(T(2) * ys[(size_t)(off + l) * R + rr] - win[(e - pd.end_off) * R + rr]);
  }
  if (a.write_x) {
    TV* xp = a.xc + (size_t)pd.copy_off * R;
    for (int i = tid; i < pd.n * R; i += kSweepThreads) xp[i] = (TV)ys[(size_t)off * R + i];
  }
}

// ------------------------------------------------------------------------------------------------
// Pipelined variant (R = 1, 2): per 32-row block step the chain warp (warp 0) finishes block k --
// the 32 columns next to the block ("near"), the partial sum prepared one step earlier ("far"), the
// inverted diagonal block -- while warps 1-7 compute the far part of block k+1 from the next slab.
// Forward: near columns [k0-32, k0), far columns < k0-32; backward (rows of U): near columns
// [k0+32, k0+64), far columns >= k0+64.  Both halves read disjoint rows of the vector, so one CTA
// barrier per block step is enough.  Needs two slabs resident (stages >= 3 keeps one in flight).
constexpr int kFarThreads = kSweepThreads - 32;
constexpr int kFarPerRow = kFarThreads / kNB;  // 7 threads per row of the next block

template <typename T, typename TV, int R>
__global__ void __launch_bounds__(kSweepThreads, 1) k_sweep_pipe(const SweepArgs<T, TV> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const PieceDesc pd = a.pieces[blockIdx.x];
  const int S = a.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  T* ring = reinterpret_cast<T*>(smem + 128);
  T* ys = ring + (size_t)S * a.slot_elems;
  T* win = ys + a.ys_elems;
  T* farp = win + a.win_elems;                        // [2][kFarPerRow][kNB][R]
  T* tbuf = farp + 2 * kFarPerRow * kNB * R;          // [kNB][R]
  constexpr int kFarBuf = kFarPerRow * kNB * R;

  const int Wp = pd.Wp;
  const int off = Wp - 1;
  const int nblk = pd.n_pad / kNB;
  const int total = 2 * nblk;
  const uint32_t slab_bytes = (uint32_t)(kNB * Wp * sizeof(T));
  const T* fbase = a.factor + pd.factor_off;
  const T* ubase = a.factor_u + pd.factor_off;

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
    bulk_copy_g2s(ring + (size_t)slot * a.slot_elems, (s < nblk ? fbase : ubase) + (size_t)kb * kNB * Wp, slab_bytes,
                  &bars[slot]);
  };
  if (tid == 0)
    for (int s = 0; s < S && s < total; ++s) issue(s);

  // ---- prologue: r_j = b̃_j + sum_e w_in[e] / Z_e at the port rows; far part of block 0 is zero
  for (int i = tid; i < off * R; i += kSweepThreads) {
    ys[i] = T(0);
    ys[(size_t)(off + pd.n_pad) * R + i] = T(0);
  }
  for (int i = tid; i < kFarBuf; i += kSweepThreads) farp[i] = T(0);
  const TV* btp = a.bt + (size_t)pd.copy_off * R;
  for (int i = tid; i < pd.n_pad * R; i += kSweepThreads) ys[(size_t)off * R + i] = (i < pd.n * R) ? (T)btp[i] : T(0);
  __syncthreads();
  for (int q = tid; q < pd.nports; q += kSweepThreads) {
    const int l = a.port_local[pd.port_off + q];
    const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
    T acc[R];
#pragma unroll
    for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
    for (int e = e0; e < e1; ++e) {
      const int tw = a.twin[e];
      const T iz = (T)a.invz[e];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const T w = (T)a.wprev[(size_t)tw * R + rr];
        win[(e - pd.end_off) * R + rr] = w;
        acc[rr] += w * iz;
      }
    }
    if (a.cpl.ptr)
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] += coupling_current<T, TV>(a.cpl, pd.port_off + q, rr, R, a.wprev);
#pragma unroll
    for (int rr = 0; rr < R; ++rr) ys[(size_t)(off + l) * R + rr] += acc[rr];
  }
  __syncthreads();

  int s = 0;
  for (; s < total; ++s) {
    const int par = s & 1;
    if (warp == 0) {
      // ---- chain: finish item s (block k0), one row per lane
      if (!mbar_wait_bounded(&bars[s % S], (uint32_t)((s / S) & 1), a.wait_limit)) abort_flag = 1;
      const T* L = ring + (size_t)(s % S) * a.slot_elems;
      const bool fwd = s < nblk;
      const int k0 = (fwd ? s : total - 1 - s) * kNB;
      const int r = lane;
      const T* Lr = L + r * Wp;
      T near[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) near[rr] = T(0);
      if (fwd) {
        const int pbeg = max(0, off - r - kNB), pend = off - r;
        const T* yb = ys + (size_t)(k0 + r) * R;
        for (int p = pbeg; p < pend; ++p) {
          const T l = Lr[p];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) near[rr] += l * yb[(size_t)p * R + rr];
        }
      } else {
        const int pbeg = kNB - r, pend = min(Wp, 2 * kNB - r);
        const T* xb = ys + (size_t)(k0 + r + off) * R;
        for (int p = pbeg; p < pend; ++p) {
          const T u = Lr[p];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) near[rr] += u * xb[(size_t)p * R + rr];
        }
      }
      const T* fp = farp + par * kFarBuf;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        T far = T(0);
#pragma unroll
        for (int h = 0; h < kFarPerRow; ++h) far += fp[(h * kNB + r) * R + rr];
        tbuf[r * R + rr] = ys[(size_t)(k0 + r + off) * R + rr] - far - near[rr];
      }
      __syncwarp();
      T y[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) y[rr] = T(0);
      if (fwd) {
        const T* Li = Lr + off - r;  // inv(L_KK)[r][c] at Li[c], c <= r
        for (int c = 0; c <= r; ++c) {
          const T l = Li[c];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) y[rr] += l * tbuf[c * R + rr];
        }
      } else {
        const T* Ui = Lr - r;        // inv(U_KK)[r][c] at Ui[c], c >= r
        for (int c = r; c < kNB; ++c) {
          const T u = Ui[c];
#pragma unroll
          for (int rr = 0; rr < R; ++rr) y[rr] += u * tbuf[c * R + rr];
        }
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr) ys[(size_t)(k0 + r + off) * R + rr] = y[rr];
    } else if (s + 1 < total) {
      // ---- far part of item s+1 from its slab (values complete at the start of step s)
      const int s1 = s + 1;
      if (!mbar_wait_bounded(&bars[s1 % S], (uint32_t)((s1 / S) & 1), a.wait_limit)) abort_flag = 1;
      const T* L1 = ring + (size_t)(s1 % S) * a.slot_elems;
      const bool fwd1 = s1 < nblk;
      const int k1 = (fwd1 ? s1 : total - 1 - s1) * kNB;
      const int t2 = tid - 32;
      const int r = t2 / kFarPerRow, h = t2 % kFarPerRow;
      const T* Lr = L1 + r * Wp;
      T acc[R];
#pragma unroll
      for (int rr = 0; rr < R; ++rr) acc[rr] = T(0);
      if constexpr (sizeof(T) == 4 && R == 1) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float4* L4 = reinterpret_cast<const float4*>(Lr);
        if (fwd1) {
          const int pend = off - r - kNB;  // far positions [0, pend)
          const float* yb = reinterpret_cast<const float*>(ys) + (k1 + r);
          for (int q = h; 4 * q < pend; q += kFarPerRow) {
            const float4 l = L4[q];
            const int p = 4 * q;
            a0 = fmaf(l.x, yb[p], a0);
            if (p + 1 < pend) a1 = fmaf(l.y, yb[p + 1], a1);
            if (p + 2 < pend) a2 = fmaf(l.z, yb[p + 2], a2);
            if (p + 3 < pend) a3 = fmaf(l.w, yb[p + 3], a3);
          }
        } else {
          const int pbeg = 2 * kNB - r;    // far positions [pbeg, Wp)
          const float* xb = reinterpret_cast<const float*>(ys) + (k1 + r + off);
          for (int q = (pbeg >> 2) + h; q < (Wp >> 2); q += kFarPerRow) {
            const float4 u = L4[q];
            const int p = 4 * q;
            if (p >= pbeg) a0 = fmaf(u.x, xb[p], a0);
            if (p + 1 >= pbeg) a1 = fmaf(u.y, xb[p + 1], a1);
            if (p + 2 >= pbeg) a2 = fmaf(u.z, xb[p + 2], a2);
            a3 = fmaf(u.w, xb[p + 3], a3);
          }
        }
        acc[0] = (a0 + a1) + (a2 + a3);
      } else {
        if (fwd1) {
          const int pend = off - r - kNB;
          const T* yb = ys + (size_t)(k1 + r) * R;
          for (int p = h; p < pend; p += kFarPerRow) {
            const T l = Lr[p];
#pragma unroll
            for (int rr = 0; rr < R; ++rr) acc[rr] += l * yb[(size_t)p * R + rr];
          }
        } else {
          const T* xb = ys + (size_t)(k1 + r + off) * R;
          for (int p = 2 * kNB - r + h; p < Wp; p += kFarPerRow) {
            const T u = Lr[p];
#pragma unroll
            for (int rr = 0; rr < R; ++rr) acc[rr] += u * xb[(size_t)p * R + rr];
          }
        }
      }
      T* fp = farp + (par ^ 1) * kFarBuf;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) fp[(h * kNB + r) * R + rr] = acc[rr];
    }
    __syncthreads();
    if (abort_flag) break;
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

  // ---- epilogue: w_out[e] = 2 x_c - w_in[e]; local solution
  for (int q = tid; q < pd.nports; q += kSweepThreads) {
    const int l = a.port_local[pd.port_off + q];
    const int e0 = a.port_end_ptr[pd.port_off + q], e1 = a.port_end_ptr[pd.port_off + q + 1];
    for (int e = e0; e < e1; ++e)
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        a.wnext[(size_t)e * R + rr] = (TV)(T(2) * ys[(size_t)(off + l) * R + rr] - win[(e - pd.end_off) * R + rr]);
  }
  if (a.write_x) {
    TV* xp = a.xc + (size_t)pd.copy_off * R;
    for (int i = tid; i < pd.n * R; i += kSweepThreads) xp[i] = (TV)ys[(size_t)off * R + i];
  }
}

size_t sweep_pipe_smem_bytes(size_t elem, int R, int stages, int slot_elems, int ys_elems, int win_elems) {
  return 128 + elem * ((size_t)stages * slot_elems + ys_elems + win_elems + (size_t)(2 * kFarPerRow + 1) * kNB * R);
}

template <typename TF, typename TV>
cudaError_t sweep_pipe_configure(int R, size_t smem) {
  switch (R) {
    case 1: return cudaFuncSetAttribute(k_sweep_pipe<TF, TV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case 2: return cudaFuncSetAttribute(k_sweep_pipe<TF, TV, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TV>
cudaError_t sweep_pipe_occupancy(int R, size_t smem, int* n) {
  switch (R) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_sweep_pipe<TF, TV, 1>, kSweepThreads, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_sweep_pipe<TF, TV, 2>, kSweepThreads, smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TV>
cudaError_t launch_sweep_pipe(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  dim3 grid(npieces), block(kSweepThreads);
  switch (R) {
    case 1: k_sweep_pipe<TF, TV, 1><<<grid, block, smem, st>>>(a); break;
    case 2: k_sweep_pipe<TF, TV, 2><<<grid, block, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t sweep_smem_bytes(size_t elem, int R, int stages, int slot_elems, int ys_elems, int win_elems) {
  return 128 + elem * ((size_t)stages * slot_elems + ys_elems + win_elems + (size_t)kNB * R);
}

template <typename TF, typename TV, int R>
static cudaError_t configure_one(size_t smem) {
  return cudaFuncSetAttribute(k_sweep<TF, TV, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename TF, typename TV>
cudaError_t sweep_configure(int R, size_t smem) {
  switch (R) {
    case 1: return configure_one<TF, TV, 1>(smem);
    case 2: return configure_one<TF, TV, 2>(smem);
    case 4: return configure_one<TF, TV, 4>(smem);
    case 8: return configure_one<TF, TV, 8>(smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TV, int R>
static cudaError_t occupancy_one(size_t smem, int* n) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_sweep<TF, TV, R>, kSweepThreads, smem);
}

template <typename TF, typename TV>
cudaError_t sweep_occupancy(int R, size_t smem, int* n) {
  switch (R) {
    case 1: return occupancy_one<TF, TV, 1>(smem, n);
    case 2: return occupancy_one<TF, TV, 2>(smem, n);
    case 4: return occupancy_one<TF, TV, 4>(smem, n);
    case 8: return occupancy_one<TF, TV, 8>(smem, n);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TF, typename TV>
cudaError_t launch_sweep(const SweepArgs<TF, TV>& a, int R, int npieces, size_t smem, cudaStream_t st) {
  if (npieces <= 0) return cudaSuccess;
  dim3 grid(npieces), block(kSweepThreads);
  switch (R) {
    case 1: k_sweep<TF, TV, 1><<<grid, block, smem, st>>>(a); break;
    case 2: k_sweep<TF, TV, 2><<<grid, block, smem, st>>>(a); break;
    case 4: k_sweep<TF, TV, 4><<<grid, block, smem, st>>>(a); break;
    case 8: k_sweep<TF, TV, 8><<<grid, block, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define VTM_SWEEP_INST(TF, TV)                                                                    \
  template cudaError_t sweep_configure<TF, TV>(int, size_t);                                       \
  template cudaError_t sweep_occupancy<TF, TV>(int, size_t, int*);                                 \
  template cudaError_t launch_sweep<TF, TV>(const SweepArgs<TF, TV>&, int, int, size_t, cudaStream_t);
VTM_SWEEP_INST(float, float)
VTM_SWEEP_INST(double, double)
VTM_SWEEP_INST(double, float)

#define VTM_PIPE_INST(TF, TV)                                                                      \
  template cudaError_t sweep_pipe_configure<TF, TV>(int, size_t);                                    \
  template cudaError_t sweep_pipe_occupancy<TF, TV>(int, size_t, int*);                               \
  template cudaError_t launch_sweep_pipe<TF, TV>(const SweepArgs<TF, TV>&, int, int, size_t, cudaStream_t);
VTM_PIPE_INST(float, float)
VTM_PIPE_INST(double, double)
VTM_PIPE_INST(double, float)

}  // namespace vtm
