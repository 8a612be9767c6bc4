// Device-side phases of the fused predistortion actor (Sec. 4.2): Poly -> FIR_k -> Adder fused into
// one dynamic actor whose control token (u32 mask, bit k = branch k active)
// is read per firing on the device.
//
// Plan kernel (one CTA per actor of a group):
//   n     = min(control tokens, data tokens, free output slots)   (all rates 1)
//   masks = the n control tokens
//   for every branch k an exclusive scan over the n firings of bit k gives
//   rank[k][i] (how many earlier firings of this step had k active) and the
//   compaction act[k][a] (firing of the a-th active block of k).  These are
//   the consumption / production counts of the internal Poly->FIR_k->Adder
//   channels, whose rate is 0 or 1 per firing.
//   The persistent history of branch k (the last MT-1 raw input samples of
//   branch k's compacted stream) is advanced into the other half of a double
//   buffer, and the channel counters are committed.
// Body kernel (persistent grid, one launch for a whole group of actors):
//   work item = (actor, firing, tile of T samples).  The x window with MT-1
//   samples of halo is staged in shared memory; per active branch the branch
//   signal z = |x|^(o-1) x is formed in a padded shared buffer (for tile 0
//   the halo comes from the branch's own history: the previous block in which
//   that branch was active, found through rank/act, or the persistent
//   history); each thread accumulates R consecutive outputs of the M-tap
//   complex FIR with the taps held in registers; the Adder is the running
//   sum over branches in registers.
#pragma once
#include <algorithm>
#include "common.cuh"

namespace dfg {


__device__ __forceinline__ float2 cmac(float2 acc, float2 h, float2 z) {
  acc.x = fmaf(h.x, z.x, acc.x);
  acc.x = fmaf(-h.y, z.y, acc.x);
  acc.y = fmaf(h.x, z.y, acc.y);
  acc.y = fmaf(h.y, z.x, acc.y);
  return acc;
}
// acc += a * conj(b)
__device__ __forceinline__ float2 cmac_conj_b(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.y, b.x, acc.y);
  acc.y = fmaf(-a.x, b.y, acc.y);
  return acc;
}

// |x|^(2q) x with u = |x|^2 raised by repeated products
__device__ __forceinline__ float2 psi_q(float2 x, int q) {
  const float u = fmaf(x.x, x.x, x.y * x.y);
  float p = 1.f;
  for (int i = 0; i < q; ++i) p *= u;
  return make_float2(p * x.x, p * x.y);
}

// ---------------------------------------------------------------- scans ----
__device__ inline uint64_t block_exclusive_scan_u64(uint64_t v, uint64_t* sw, uint64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t s = lane < nw ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sw[lane] = s;
  }
  __syncthreads();
  const uint64_t before = wid ? sw[wid - 1] : 0;
  *total = sw[nw - 1];
  __syncthreads();
  return before + x - v;
}

// ------------------------------------------------------------ FIR cores ----
// Shared windows are padded with one element after every R elements so that
// threads reading at stride R elements hit distinct banks.
// Causal chunk: acc[r] += sum_{m<MC} h[m] * zs[v], v = p*R + shift + r - m + MC - 1.
// Taps m >= m_valid are zero (unpadded tap rows).  The complex product is
// issued as two passes over the R outputs (real tap part, then imaginary tap
// part) so consecutive FMAs update different accumulators.
template <int R, int MC>
__device__ __forceinline__ void fir_causal(float2 (&acc)[R], const float2* __restrict__ zs, int p,
                                           int shift, const float2* __restrict__ h, int m_valid) {
  float2 hk[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) hk[m] = m < m_valid ? h[m] : make_float2(0.f, 0.f);
  const float2* zb = zs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const float2 z = zb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) {
        acc[r].x = fmaf(hk[m].x, z.x, acc[r].x);
        acc[r].y = fmaf(hk[m].x, z.y, acc[r].y);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) {
        acc[r].x = fmaf(-hk[m].y, z.y, acc[r].x);
        acc[r].y = fmaf(hk[m].y, z.x, acc[r].y);
      }
    }
  }
}

// Anti-causal chunk with conjugated taps: acc[r] += sum_m conj(h[m]) * gs[v], v = p*R + shift + r + m.
template <int R, int MC>
__device__ __forceinline__ void fir_anticausal_conj(float2 (&acc)[R], const float2* __restrict__ gs,
                                                    int p, int shift, const float2* __restrict__ h,
                                                    int m_valid) {
  float2 ck[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const float2 t = m < m_valid ? __ldg(h + m) : make_float2(0.f, 0.f);
    ck[m] = make_float2(t.x, -t.y);
  }
  const float2* gb = gs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const float2 g = gb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = s - r;
      if (m >= 0 && m < MC) acc[r] = cmac(acc[r], ck[m], g);
    }
  }
}

// Tap-gradient chunk: ph[m] += sum_r g[r] * conj(zs[v]), v = p*R + shift + r - m + MC - 1.
template <int R, int MC>
__device__ __forceinline__ void gh_chunk(float2 (&ph)[MC], const float2 (&gr)[R],
                                         const float2* __restrict__ zs, int p, int shift) {
  const float2* zb = zs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const float2 z = zb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) ph[m] = cmac_conj_b(ph[m], gr[r], z);
    }
  }
}

// FIR of one branch over a staged window, MT <= 16 in one chunk, MT == 32 in two.
// h points at the M valid taps of the branch (M <= MT).
template <int R, int MT>
__device__ __forceinline__ void fir_branch(float2 (&acc)[R], const float2* zs, int p,
                                           const float2* h, int M) {
  if constexpr (MT <= 16) {
    fir_causal<R, MT>(acc, zs, p, 0, h, M);
  } else {
    fir_causal<R, 16>(acc, zs, p, 16, h, M);
    fir_causal<R, 16>(acc, zs, p, 0, h + 16, M - 16);
  }
}

// Packed form for the body kernel: two-lane FMAs (one instruction updates
// the real and imaginary parts).  With taps staged as {hx, hx, hy, hy}, the
// output is split into A = sum hx * z and B = sum hy * z (both lanes of z), so
// that every product has the same tap value in both lanes; the complex result
// is (A.x - B.y, A.y + B.x), formed once after all branches.
template <int R, int MC>
__device__ __forceinline__ void fir_causal_x2(float2 (&A)[R], float2 (&B)[R], const float2* __restrict__ zs,
                                              int p, int shift, const float4* __restrict__ h4,
                                              int m_valid) {
  float2 hxx[MC], hyy[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const float4 t = m < m_valid ? h4[m] : make_float4(0.f, 0.f, 0.f, 0.f);
    hxx[m] = make_float2(t.x, t.y);
    hyy[m] = make_float2(t.z, t.w);
  }
  const float2* zb = zs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const float2 z = zb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) {
        A[r] = __ffma2_rn(hxx[m], z, A[r]);
        B[r] = __ffma2_rn(hyy[m], z, B[r]);
      }
    }
  }
}

template <int R, int MT>
__device__ __forceinline__ void fir_branch_x2(float2 (&A)[R], float2 (&B)[R], const float2* zs, int p,
                                              const float4* h4, int M) {
  if constexpr (MT <= 16) {
    fir_causal_x2<R, MT>(A, B, zs, p, 0, h4, M);
  } else {
    fir_causal_x2<R, 16>(A, B, zs, p, 16, h4, M);
    fir_causal_x2<R, 16>(A, B, zs, p, 0, h4 + 16, M - 16);
  }
}

#define DPD_MT_CASES(X) X(4) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(32)

// ----------------------------------------------------------------- plan ----
__device__ inline void dpd_plan_dev(const DpdArgs& a) {
  __shared__ uint64_t s_n, s_rdc, s_rdd, s_wro;
  __shared__ uint32_t s_par;
  __shared__ uint64_t sw[32];
  uint64_t* ctr = a.ctr;
  const bool has_ctrl = a.ctrl.ring != nullptr;
  if (threadIdx.x == 0) {
    const uint64_t rdc = has_ctrl ? *rd_ptr(ctr, a.ctrl.id) : 0;
    const uint64_t wrc = has_ctrl ? *wr_ptr(ctr, a.ctrl.id) : ~0ull;
    const uint64_t rdd = *rd_ptr(ctr, a.data.id), wrd = *wr_ptr(ctr, a.data.id);
    const uint64_t wro = *wr_ptr(ctr, a.out.id), rdo = *rd_ptr(ctr, a.out.id);
    uint64_t n = wrc - rdc;
    n = min(n, wrd - rdd);
    n = min(n, a.out.cap - (wro - rdo));
    n = min(n, (uint64_t)a.n_max);
    s_n = n; s_rdc = rdc; s_rdd = rdd; s_wro = wro; s_par = *a.parity;
  }
  __syncthreads();
  const uint32_t n = (uint32_t)s_n;
  const uint32_t kmask = a.K >= 32 ? 0xffffffffu : ((1u << a.K) - 1u);
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
    a.masks[i] = has_ctrl ? *reinterpret_cast<const uint32_t*>(slot_ptr(a.ctrl, s_rdc + i)) & kmask
                          : kmask;
  __syncthreads();
  for (int k = 0; k < a.K; ++k) {
    uint64_t carry = 0;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
      const uint32_t i = base + threadIdx.x;
      const uint32_t bit = i < n ? (a.masks[i] >> k) & 1u : 0u;
      uint64_t tot;
      const uint64_t ex = block_exclusive_scan_u64(bit, sw, &tot);
      if (i < n) {
        a.rank[(size_t)k * a.n_max + i] = (uint32_t)(carry + ex);
        if (bit) a.act[(size_t)k * a.n_max + carry + ex] = i;
      }
      carry += tot;
    }
    if (threadIdx.x == 0) a.cnt[k] = (uint32_t)carry;
  }
  __syncthreads();
  const int H1 = a.MT - 1;
  if (n > 0 && H1 > 0) {
    const uint32_t par = s_par;
    for (int e = threadIdx.x; e < a.K * H1; e += blockDim.x) {
      const int k = e / H1, s = e % H1;
      const int64_t pos = (int64_t)a.cnt[k] * a.L - H1 + s;
      float2 v;
      if (pos >= 0) {
        const uint32_t f = a.act[(size_t)k * a.n_max + (uint32_t)(pos / a.L)];
        v = reinterpret_cast<const float2*>(slot_ptr(a.data, s_rdd + f))[pos % a.L];
      } else {
        v = a.hist[((size_t)par * a.K + k) * H1 + (H1 + pos)];
      }
      a.hist[((size_t)(par ^ 1) * a.K + k) * H1 + s] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.plan->n = n;
    a.plan->rd_data0 = s_rdd;
    a.plan->wr_out0 = s_wro;
    a.plan->slot_data0 = s_rdd % a.data.cap;
    a.plan->slot_out0 = (s_wro - a.out.wshift) % a.out.cap;
    a.plan->parity_in = s_par;
    if (n > 0) *a.parity = s_par ^ 1u;
    if (has_ctrl) *rd_ptr(ctr, a.ctrl.id) = s_rdc + n;
    *rd_ptr(ctr, a.data.id) = s_rdd + n;
    *wr_ptr(ctr, a.out.id) = s_wro + n;
    atomicAdd(&a.eng->fired_total, (unsigned long long)n);
  }
}

// ----------------------------------------------------------------- body ----
__device__ __forceinline__ float2 hist_sample(const DpdArgs& a, const DpdPlanHdr& pl, uint32_t i,
                                              int k, int s) {
  const int H1 = a.MT - 1;
  const int64_t pos = (int64_t)a.rank[(size_t)k * a.n_max + i] * a.L - H1 + s;
  if (pos >= 0) {
    const uint32_t f = a.act[(size_t)k * a.n_max + (uint32_t)(pos / a.L)];
    return reinterpret_cast<const float2*>(slot_ptr(a.data, pl.rd_data0 + f))[pos % a.L];
  }
  return a.hist[((size_t)pl.parity_in * a.K + k) * H1 + (H1 + pos)];
}

constexpr int kBranchGroup = 1;           // branch signals staged at once

// u^q from the squares u, u^2, u^4, u^8 (q < 16), else by repeated products.
__device__ __forceinline__ float pow_sq(float u, float u2, float u4, float u8, int q) {
  if (q >= 16) {
    float p = 1.f;
    for (int i = 0; i < q; ++i) p *= u;
    return p;
  }
  float p = (q & 1) ? u : 1.f;
  if (q & 2) p *= u2;
  if (q & 4) p *= u4;
  if (q & 8) p *= u8;
  return p;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ const uint8_t* slot_at(const ChanDesc& c, uint64_t slot0, uint32_t i) {
  uint64_t s = slot0 + i;
  if (s >= c.cap) s -= c.cap;
  return c.ring + s * c.tok;
}

struct ItemRef {
  int g;                    // actor within the group, -1 = none
  uint32_t i;               // firing
  uint32_t t0;              // first sample of the tile
  int len;                  // samples of the tile inside the block
};

__device__ __forceinline__ ItemRef locate(const DpdArgs* args, const uint64_t* s_off, int G,
                                          uint64_t item, uint64_t total, uint32_t T) {
  ItemRef r{-1, 0, 0, 0};
  if (item >= total) return r;
  int lo = 0, hi = G;                     // s_off[lo] <= item < s_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_off[mid] <= item) lo = mid; else hi = mid;
  }
  const DpdArgs& a = args[lo];
  const uint64_t local = item - s_off[lo];
  const uint32_t nt = (a.L + T - 1) / T;
  r.g = lo;
  r.i = (uint32_t)(local / nt);
  r.t0 = (uint32_t)(local % nt) * T;
  r.len = (int)min(T, a.L - r.t0);
  return r;
}

// Copy the x window of `it` (x[t0 - (MT-1) .. t0 + T), zeros outside the block) into xs.
__device__ __forceinline__ void prefetch_x(const DpdArgs& a, const ItemRef& it, float2* xs, uint32_t T) {
  const DpdPlanHdr* pl = a.plan;
  const float2* xb = reinterpret_cast<const float2*>(slot_at(a.data, pl->slot_data0, it.i)) + it.t0;
  const int MT = a.MT;
  const int W = (int)T + MT - 1;
  for (int v = threadIdx.x; v < W; v += blockDim.x) {
    const int pos = v - (MT - 1);
    const bool valid = pos < it.len && (int)it.t0 + pos >= 0;
    cp_async8(xs + v, valid ? (const void*)(xb + pos) : (const void*)xb, valid);
  }
}

// u^Q by a fixed multiplication chain (Q known at compile time).
template <int Q>
__device__ __forceinline__ float pow_c(float u) {
  if constexpr (Q == 0) {
    return 1.f;
  } else if constexpr (Q == 1) {
    return u;
  } else if constexpr (Q % 2 == 0) {
    const float h = pow_c<Q / 2>(u);
    return h * h;
  } else {
    return pow_c<Q - 1>(u) * u;
  }
}

// zg[v + v/R] = |x_v|^(2Q) x_v for the window v < W (padded layout).
template <int R, int Q>
__device__ __forceinline__ void zpass(const float2* __restrict__ xs, float2* __restrict__ zg, int W) {
  const int P = blockDim.x;
#pragma unroll 4
  for (int v = threadIdx.x; v < W; v += P) {
    const float2 x = xs[v];
    const float pw = pow_c<Q>(fmaf(x.x, x.x, x.y * x.y));
    zg[v + v / R] = make_float2(pw * x.x, pw * x.y);
  }
}

template <int R>
__device__ inline void zpass_any(const float2* __restrict__ xs, float2* __restrict__ zg, int W, int q) {
  for (int v = threadIdx.x; v < W; v += blockDim.x) zg[v + v / R] = psi_q(xs[v], q);
}

// Shared memory of one body CTA (T = R * blockDim.x samples per tile, W = T + MTmax - 1):
//   xs[2][W] float2 | zb[kBranchGroup][Wp] float2 (Wp = W + W / R + 2) |
//   hs[kMaxBranches * MTmax] float4 {hx, hx, hy, hy}
template <int R, int MT>
__device__ inline void dpd_compute(const DpdArgs& a, const ItemRef& it, const float2* xs, float2* zb,
                            int Wp, const float4* hs, int* s_k, int* s_q) {
  const int P = blockDim.x, p = threadIdx.x;
  const uint32_t T = R * P;
  const DpdPlanHdr& pl = *a.plan;
  const uint32_t mask = a.masks[it.i];
  float2* yb = reinterpret_cast<float2*>(const_cast<uint8_t*>(slot_at(a.out, pl.slot_out0, it.i))) + it.t0;
  if (mask == 0) {
    for (int o = p; o < it.len; o += P) yb[o] = make_float2(0.f, 0.f);
    return;
  }
  const int W = (int)T + MT - 1;
  int nk = 0;
  {
    uint32_t rest = mask;
    while (rest) {
      const int k = __ffs(rest) - 1;
      rest &= rest - 1;
      if (p == 0) {
        s_k[nk] = k;
        s_q[nk] = (a.orders[k] - 1) >> 1;
      }
      ++nk;
    }
  }
  __syncthreads();
  float2 A[R], B[R];                      // sums of hx * z and hy * z (see fir_causal_x2)
#pragma unroll
  for (int r = 0; r < R; ++r) A[r] = B[r] = make_float2(0.f, 0.f);
  for (int g0 = 0; g0 < nk; g0 += kBranchGroup) {
    const int ng = min(kBranchGroup, nk - g0);
    // branch signals z = u^q x of this group for the whole window, one tight loop per branch
    for (int g = 0; g < ng; ++g) {
      float2* zg = zb + g * Wp;
      switch (s_q[g0 + g]) {
#define ZP(Q) case Q: zpass<R, Q>(xs, zg, W); break;
        ZP(0) ZP(1) ZP(2) ZP(3) ZP(4) ZP(5) ZP(6) ZP(7)
        ZP(8) ZP(9) ZP(10) ZP(11) ZP(12) ZP(13) ZP(14) ZP(15)
#undef ZP
        default: zpass_any<R>(xs, zg, W, s_q[g0 + g]); break;
      }
    }
    if (it.t0 == 0) {
      // tile 0: the MT-1 samples before the block come from each branch's own history
      for (int e = p; e < ng * (MT - 1); e += P) {
        const int g = e / (MT - 1), v = e - g * (MT - 1);
        zb[g * Wp + v + v / R] = psi_q(hist_sample(a, pl, it.i, s_k[g0 + g], v), s_q[g0 + g]);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < ng; ++g) fir_branch_x2<R, MT>(A, B, zb + g * Wp, p, hs + s_k[g0 + g] * MT, MT);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) zb[p * (R + 1) + r] = make_float2(A[r].x - B[r].y, A[r].y + B[r].x);
  __syncthreads();
  for (int o = p; o < it.len; o += P) yb[o] = zb[o + o / R];
}

constexpr int kMaxGroup = 1024;

template <int R, int MTMAX>
__device__ inline void dpd_body_dev(const DpdArgs* __restrict__ args, int G, Grid grid,
                                    float4* smem_raw) {
  __shared__ uint64_t sw[32];
  __shared__ int s_k[kMaxBranches], s_q[kMaxBranches];
  const uint32_t T = R * blockDim.x;
  const int Wm = (int)T + MTMAX - 1;
  const int Wpm = Wm + Wm / R + 2;
  // taps (float4, 16-byte aligned) follow the tile buffers; then the work-list
  // offsets of the group's actors
  const int hs_off = (2 * Wm + kBranchGroup * Wpm + 1) & ~1;          // in float2 units
  uint64_t* s_off = reinterpret_cast<uint64_t*>(reinterpret_cast<float2*>(smem_raw) + hs_off +
                                                2 * kMaxBranches * MTMAX);
  uint64_t carry = 0;
  for (int base = 0; base < G; base += blockDim.x) {
    const int g = base + threadIdx.x;
    uint64_t items = 0;
    if (g < G) {
      const DpdArgs& a = args[g];
      items = a.plan->n * ((a.L + T - 1) / T);
    }
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan_u64(items, sw, &tot);
    if (g < G) s_off[g] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) s_off[G] = carry;
  __syncthreads();
  const uint64_t total = carry;
  const int W = (int)T + MTMAX - 1;
  const int Wp = W + W / R + 2;
  float2* xsb = reinterpret_cast<float2*>(smem_raw);          // [2][W]
  float2* zb = xsb + 2 * W;
  float4* hs = reinterpret_cast<float4*>(xsb + hs_off);              // taps {hx, hx, hy, hy}
  int taps_of = -1;                                            // actor whose taps are in hs
  uint64_t item = grid.b;
  ItemRef cur = locate(args, s_off, G, item, total, T);
  if (cur.g >= 0) prefetch_x(args[cur.g], cur, xsb, T);
  cp_async_commit();
  int buf = 0;
  while (cur.g >= 0) {
    const uint64_t next_item = item + grid.n;
    const ItemRef nxt = locate(args, s_off, G, next_item, total, T);
    if (nxt.g >= 0) prefetch_x(args[nxt.g], nxt, xsb + (buf ^ 1) * W, T);
    cp_async_commit();
    if (cur.g != taps_of) {
      const DpdArgs& a = args[cur.g];
      for (int e = threadIdx.x; e < a.K * a.MT; e += blockDim.x) {
        const float2 h = a.h[e];
        hs[e] = make_float4(h.x, h.x, h.y, h.y);
      }
      taps_of = cur.g;
    }
    cp_async_wait1();
    __syncthreads();
    const DpdArgs& a = args[cur.g];
    switch (a.MT) {
#define DPD_CASE(MTV) \
      case MTV: if constexpr (MTV <= MTMAX) dpd_compute<R, MTV>(a, cur, xsb + buf * W, zb, Wp, hs, s_k, s_q); break;
      DPD_MT_CASES(DPD_CASE)
#undef DPD_CASE
      default: break;
    }
    __syncthreads();
    cur = nxt;
    item = next_item;
    buf ^= 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace dfg
