// Device-side phases of the fused predistortion actor (Sec. 4.2): Poly -> FIR_k -> Adder fused into
// one dynamic actor whose control token (u32 mask, bit k = branch k active)
// is read per firing on the device.
//
// Plan kernel (one CTA per actor of a group):
//   n     = min(control tokens, data tokens, free output slots)   (all rates 1)
//   masks = the n control tokens
//   for every branch k an exclusive scan over the n firings of bit k gives
//   rank[k][i] (how many earlier firings of this step had k active), the
//   compaction act[k][a] (firing of the a-th active block of k) and
//   prev[k][i] (the latest earlier firing with k active, -1: none).  These are
//   the consumption / production counts of the internal Poly->FIR_k->Adder
//   channels, whose rate is 0 or 1 per firing.
//   The channel counters are committed.  The persistent history of branch k
//   (the last MT-1 raw input samples of branch k's compacted stream) is
//   advanced into the other half of a double buffer by the body kernel, off
//   the step's critical path.
// Body kernel (one launch for a whole group of actors, a grid sized to the
//   SMs): work item = (actor, firing, chunk of 32 R output samples), taken by
//   one warp.  The x window with MT-1 samples of halo is staged in the warp's
//   shared memory; per active branch the branch signal z = |x|^(o-1) x is
//   formed in a padded shared buffer (for a block's first chunk the halo comes
//   from the branch's own history: the previous block in which that branch
//   was active, found through rank/act, or the persistent history); each lane
//   accumulates R consecutive outputs of the M-tap complex FIR with the taps in
//   registers; the Adder is the running sum over branches in registers.
#pragma once
#include <algorithm>
#include "common.cuh"

namespace dfg {


// u^q for a runtime q, by squaring
__device__ __forceinline__ float upow(float u, int q) {
  float p = (q & 1) ? u : 1.f;
  for (int e = q >> 1; e; e >>= 1) {
    u *= u;
    if (e & 1) p *= u;
  }
  return p;
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

#define DPD_MT_CASES(X) X(4) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(32)

// ----------------------------------------------------------------- plan ----
// The plan decides the step and commits it; the persistent history it leaves
// for the next step is advanced later, beside the body (dpd_hist_dev), since
// this step's body does not read it.
__device__ inline void dpd_plan_dev(const DpdArgs& a) {
  __shared__ uint64_t s_n, s_rdc, s_rdd, s_wro;
  __shared__ uint32_t s_par;
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
  // Per branch k, the exclusive scan of its activity bits over the firings:
  // one warp per branch (branches dealt round-robin to the warps), 32
  // firings per ballot, each warp reading the control tokens itself, so no
  // barrier separates reading them from the scans.  The warp of branch 0
  // also stores the masks for the body.
  {
    const int lane = threadIdx.x & 31, nwarp = (int)(blockDim.x >> 5);
    const uint32_t below = (1u << lane) - 1u;
    for (int k = (int)(threadIdx.x >> 5); k < a.K; k += nwarp) {
      uint32_t carry = 0;
      int last = -1;
      for (uint32_t base = 0; base < n; base += 32) {
        const uint32_t i = base + lane;
        uint32_t m = 0;
        if (i < n)
          m = has_ctrl ? *reinterpret_cast<const uint32_t*>(slot_ptr(a.ctrl, s_rdc + i)) & kmask : kmask;
        if (k == 0 && i < n) a.masks[i] = m;
        const bool bit = (m >> k) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, bit);
        const uint32_t bb = b & below;
        const uint32_t ex = carry + __popc(bb);
        if (i < n) {
          a.rank[(size_t)k * a.n_max + i] = ex;
          a.prev[(size_t)k * a.n_max + i] = bb ? (int)base + 31 - __clz(bb) : last;
          if (bit) a.act[(size_t)k * a.n_max + ex] = i;
        }
        carry += __popc(b);
        if (b) last = (int)base + 31 - __clz(b);
      }
      if (lane == 0) {
        a.cnt[k] = carry;
        a.plan->last[k] = last;
      }
    }
  }
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

// The persistent history of every branch after this step (the last MT-1
// samples of its compacted input stream) into the other half of the double
// buffer: the tail of the latest active firing, else the history carried in.
// Runs by one CTA after the plan, beside or after the body (which reads only
// the half the plan named), and before the next step's plan.
__device__ inline void dpd_hist_dev(const DpdArgs& a) {
  const DpdPlanHdr& pl = *a.plan;
  const uint32_t n = (uint32_t)pl.n;
  const int H1 = a.MT - 1;
  if (n == 0 || H1 <= 0) return;
  const uint32_t par = pl.parity_in;
  for (int e = threadIdx.x; e < a.K * H1; e += blockDim.x) {
    const int k = e / H1, s = e % H1;
    float2 v;
    if ((uint32_t)H1 <= a.L) {
      const int f = pl.last[k];
      v = f >= 0 ? reinterpret_cast<const float2*>(slot_ptr(a.data, pl.rd_data0 + (uint32_t)f))[a.L - H1 + s]
                 : a.hist[((size_t)par * a.K + k) * H1 + s];
    } else {
      // history longer than a block: it spans several earlier firings
      const int64_t pos = (int64_t)a.cnt[k] * a.L - H1 + s;
      if (pos >= 0) {
        const uint32_t f = a.act[(size_t)k * a.n_max + (uint32_t)(pos / a.L)];
        v = reinterpret_cast<const float2*>(slot_ptr(a.data, pl.rd_data0 + f))[pos % a.L];
      } else {
        v = a.hist[((size_t)par * a.K + k) * H1 + (H1 + pos)];
      }
    }
    a.hist[((size_t)(par ^ 1) * a.K + k) * H1 + s] = v;
  }
}

// ----------------------------------------------------------------- body ----
// The body is warp-granular: a work item is (actor, firing, chunk of 32 * R
// consecutive output samples of the block), and every warp walks its own
// items with its own shared memory, so no barrier spans more than one warp
// after the kernel's start.  Items are dealt to warps interleaved across the
// CTAs of the grid (warp w of CTA b is global warp w * gridDim + b), so
// neighbouring chunks run on different SMs at the same time.
//
// Per item: the x window x[t0 - (MT-1) .. t0 + 32R) of the block (zeros
// outside it) is staged by cp.async into one half of a double buffer while
// the previous item computes.  Per active branch k, in ascending k:
//   z-pass: lane l forms z = |x|^(o_k - 1) x for window positions l, l + 32,
//           ..., stored as {zx, zy} (the first MT-1 positions of a block's
//           first chunk come from branch k's own history instead: the
//           previous block in which k was active, or the persisted history);
//   FIR:    lane l loads its R + MT - 1 window positions of z into registers
//           and accumulates outputs l*R .. l*R + R-1 tap by tap, each tap
//           {hx, hx, hy, hy} one 16-byte shared load at the same address in
//           every lane, with two-lane FMAs P += {zx, zy} * {hx, hx} and
//           Q += {zx, zy} * {hy, hy}, so that y = (P.x - Q.y, P.y + Q.x) is
//           the complex sum over taps and branches (the Adder), formed once
//           at the end.
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

// Shared memory of one warp (R outputs per lane, taps padded to at most MTMAX):
//   xw[2][XW] float2  x window, double buffered (XW >= 32 (R + 1) and >= 32R + MTMAX - 1, even)
//   zw[ZW]    float2  branch signal {zx, zy}; position v at v + v / R, so
//                     that the 16 lanes of a half-warp reading at a stride of
//                     R positions hit distinct banks
//   hw[kMaxBranches * MTMAX] float4  taps {hx, hx, hy, hy} of the warp's
//                     current actor, then its branch orders (int32)
//   mw[2] u32         control masks of the two buffered items (staged with x)
template <int R, int MTMAX>
struct WarpSmem {
  static constexpr int XW = 32 * (R + 1) > 32 * R + MTMAX - 1 ? 32 * (R + 1) : ((32 * R + MTMAX) & ~1);
  static constexpr int ZW = (XW + XW / R + 2) & ~1;
  static constexpr size_t x_bytes = 2 * (size_t)XW * sizeof(float2);
  static constexpr size_t z_bytes = (size_t)ZW * sizeof(float2);
  static constexpr size_t h_bytes = (size_t)kMaxBranches * MTMAX * sizeof(float4) + kMaxBranches * sizeof(int32_t);
  static constexpr size_t m_bytes = 16;     // control masks of the two buffered items
  static constexpr size_t bytes = x_bytes + z_bytes + h_bytes + m_bytes;
};

// Bytes before the per-warp areas: the work-list offsets of G actors and
// their visiting order.
__host__ __device__ constexpr size_t dpd_body_off_bytes(int G) {
  return ((size_t)(G + 1) * sizeof(uint64_t) + (size_t)G * sizeof(uint16_t) + 15) & ~(size_t)15;
}

template <int R, int MTMAX>
__host__ __device__ constexpr size_t dpd_body_smem(int warps, int G) {
  return dpd_body_off_bytes(G) + (size_t)warps * WarpSmem<R, MTMAX>::bytes;
}

struct WItem {
  int g;                    // actor within the group, -1 = none
  uint32_t i;               // firing
  uint32_t t0;              // first sample of the chunk
  int len;                  // samples of the chunk inside the block
  int shift;                // staged window starts this many elements into its buffer
};

// Where item `item` of the group's work list is: a binary search over the
// actors' first items, then firing and chunk by division.  The warp's last
// answer is kept (LocHint): the next item of a run is the next chunk of the
// same block or the first chunk of the next firing, and an item in the same
// actor needs no search.
struct LocHint {
  int lo = -1;                  // position in the ordered actor list, -1: none
  int g = -1;
  uint32_t nt = 0, L = 0;       // chunks per block, samples per block
  uint64_t beg = 0, end = 0;    // the actor's items [beg, end)
  uint64_t item = ~0ull;        // last item located
  uint32_t i = 0, t0 = 0;       // its firing and first sample
};

__device__ __forceinline__ WItem locate_w(const DpdArgs* args, const uint64_t* s_off, const uint16_t* s_ord,
                                          int G, uint64_t item, uint64_t total, uint32_t WI, LocHint& h) {
  WItem r{-1, 0, 0, 0, 0};
  if (item >= total) return r;
  if (h.lo >= 0 && item == h.item + 1 && item < h.end) {
    h.t0 += WI;
    if (h.t0 >= h.L) {
      h.t0 = 0;
      ++h.i;
    }
  } else {
    if (h.lo < 0 || item < h.beg || item >= h.end) {
      int lo = 0, hi = G;                     // s_off[lo] <= item < s_off[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_off[mid] <= item) lo = mid; else hi = mid;
      }
      h.lo = lo;
      h.g = s_ord[lo];
      h.L = args[h.g].L;
      h.nt = (h.L + WI - 1) / WI;
      h.beg = s_off[lo];
      h.end = s_off[lo + 1];
    }
    const uint64_t local = item - h.beg;
    if (local < 0xffffffffull) {
      const uint32_t l32 = (uint32_t)local;
      h.i = l32 / h.nt;
      h.t0 = (l32 - h.i * h.nt) * WI;
    } else {
      h.i = (uint32_t)(local / h.nt);
      h.t0 = (uint32_t)(local % h.nt) * WI;
    }
  }
  h.item = item;
  r.g = h.g;
  r.i = h.i;
  r.t0 = h.t0;
  r.len = (int)min(WI, h.L - h.t0);
  return r;
}

// Stage the x window of `it` into the buffer xb0 (position v holds sample
// t0 - (MT-1) + v of the block, zero outside [0, t0 + len)) and its control
// mask into mask_dst.  The window is copied as 16-byte pairs of samples from
// the first 16-byte boundary at or before its start, so that every copy but
// the edge pairs is a 16-byte one; it.shift records where position 0 landed.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void prefetch_w(const DpdArgs& a, WItem& it, float2* xb0, uint32_t* mask_dst,
                                           uint32_t WI, int lane) {
  const DpdPlanHdr* pl = a.plan;
  const float2* xb = reinterpret_cast<const float2*>(slot_at(a.data, pl->slot_data0, it.i));
  const int H1 = a.MT - 1;
  const int W = (int)WI + H1;
  const int end = (int)it.t0 + it.len;
  const int pos0 = (int)it.t0 - H1;
  const int par = (reinterpret_cast<uintptr_t>(xb) & 15) == 0 ? 0 : 1;   // sample indices on a 16-byte boundary
  const int a0 = pos0 - ((pos0 - par) & 1);
  it.shift = pos0 - a0;
  const int npairs = (W + it.shift + 1) / 2;
  for (int p = lane; p < npairs; p += 32) {
    const int idx = a0 + 2 * p;
    const bool v0 = idx >= 0 && idx < end, v1 = idx + 1 >= 0 && idx + 1 < end;
    if (v0 && v1) {
      cp_async16(xb0 + 2 * p, xb + idx);
    } else {
      cp_async8(xb0 + 2 * p, v0 ? (const void*)(xb + idx) : (const void*)xb, v0);
      cp_async8(xb0 + 2 * p + 1, v1 ? (const void*)(xb + idx + 1) : (const void*)xb, v1);
    }
  }
  if (lane == 0) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(mask_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(a.masks + it.i) : "memory");
  }
}

__device__ __forceinline__ void zstore(float2* zw, int v, int R, float2 x, float p) {
  zw[v + v / R] = make_float2(p * x.x, p * x.y);
}

// z = u^q x over all 32 (R + 1) window positions lane, lane + 32, ...; the x
// and z buffers hold that many, positions >= W hold stale x and are never
// used by the FIR, so the pass is straight-line code: all loads, then the
// arithmetic, then all stores.  Position lane + 32 j of the padded z buffer
// sits at lane + lane / R + j (32 + 32 / R) (R divides 32): fixed offsets from
// one per-lane base.  u^q is assembled from u, u^2 and u^4 by the bits of q
// (q < 8, orders up to 15), by repeated products otherwise.
template <int R>
__device__ __forceinline__ void zpass_w(const float2* __restrict__ xs, float2* __restrict__ zw, int lane, int q) {
  const float2* xb = xs + lane;
  float2* zb = zw + lane + lane / R;
  float2 x[R + 1];
#pragma unroll
  for (int j = 0; j <= R; ++j) x[j] = xb[32 * j];
  float p[R + 1];
  if (q < 8) {
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      const float u = fmaf(x[j].x, x[j].x, x[j].y * x[j].y);
      const float u2 = u * u;
      float v = (q & 1) ? u : 1.f;
      if (q & 2) v *= u2;
      if (q & 4) v *= u2 * u2;
      p[j] = v;
    }
  } else {
#pragma unroll
    for (int j = 0; j <= R; ++j) {
      const float u = fmaf(x[j].x, x[j].x, x[j].y * x[j].y);
      float v = 1.f;
      for (int e = 0; e < q; ++e) v *= u;
      p[j] = v;
    }
  }
#pragma unroll
  for (int j = 0; j <= R; ++j) {
    zb[j * (32 + 32 / R)] = make_float2(p[j] * x[j].x, p[j] * x[j].y);
  }
}

// Two-lane FP32 FMA on 64-bit registers holding a pair of floats (element 0 in
// the low half): d = a * b + d elementwise.  Keeping the operands in 64-bit
// registers end to end means no register pairs have to be formed around the
// instruction.
__device__ __forceinline__ void ffma2_b64(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 unpack_b64(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// One branch's FIR into the accumulators of this lane's R outputs:
// P[r] += {zx, zy} * {hx, hx}, Q[r] += {zx, zy} * {hy, hy} over the MT taps.
template <int R, int MT>
__device__ __forceinline__ void fir_w(unsigned long long (&P)[R], unsigned long long (&Q)[R],
                                      const float2* __restrict__ zw, int lane, const ulonglong2* __restrict__ hk) {
  // the lane's R + MT - 1 window positions {zx, zy}, then tap by tap
  const unsigned long long* zb = reinterpret_cast<const unsigned long long*>(zw) + lane * (R + 1);
  unsigned long long z[R + MT - 1];
#pragma unroll
  for (int s = 0; s < R + MT - 1; ++s) z[s] = zb[s + s / R];
#pragma unroll
  for (int m = 0; m < MT; ++m) {
    const ulonglong2 h = hk[m];                // {hx, hx}, {hy, hy}: one address for the warp
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ffma2_b64(P[r], z[r + MT - 1 - m], h.x);
      ffma2_b64(Q[r], z[r + MT - 1 - m], h.y);
    }
  }
}

// Outputs o = lane*R + r of the chunk (o < len) at yb.
template <int R>
__device__ __forceinline__ void store_w(float2* yb, int len, int lane, const float2 (&y)[R]) {
  const int o0 = lane * R;
  if (len == 32 * R && (reinterpret_cast<uintptr_t>(yb) & 15) == 0) {
#pragma unroll
    for (int r = 0; r < R; r += 2)
      *reinterpret_cast<float4*>(yb + o0 + r) = make_float4(y[r].x, y[r].y, y[r + 1].x, y[r + 1].y);
  } else if (len == 32 * R) {
    // 8 bytes off a 16-byte boundary (a block of odd length in every other
    // ring slot): one sample, 16-byte pairs, one sample
    yb[o0] = y[0];
#pragma unroll
    for (int r = 1; r < R - 1; r += 2)
      *reinterpret_cast<float4*>(yb + o0 + r) = make_float4(y[r].x, y[r].y, y[r + 1].x, y[r + 1].y);
    yb[o0 + R - 1] = y[R - 1];
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (o0 + r < len) yb[o0 + r] = y[r];
  }
}

// One work item.  A block's first chunk also needs, per active branch, the
// MT-1 samples before the block in that branch's stream: the tail of the
// latest earlier firing of this step with the branch active (prev, from the
// plan), else the persisted history; blocks shorter than MT-1 samples take
// them from several earlier firings (hist_sample).
template <int R, int MT>
__device__ __noinline__ void dpd_item_w(const DpdArgs& a, const WItem& it, uint32_t mask, const float2* xs,
                                        float2* zw, const ulonglong2* hw, int lane) {
  const DpdPlanHdr& pl = *a.plan;
  float2* yb = reinterpret_cast<float2*>(const_cast<uint8_t*>(slot_at(a.out, pl.slot_out0, it.i))) + it.t0;
  unsigned long long P[R], Q[R];              // pairs of floats, +0.0f each
#pragma unroll
  for (int r = 0; r < R; ++r) P[r] = Q[r] = 0ull;
  const int32_t* ok = reinterpret_cast<const int32_t*>(hw + a.K * MT);   // branch orders
  const bool first = it.t0 == 0;
  const bool short_block = a.L < (uint32_t)(MT - 1);
  int pv = -1;                                // lane k: prev[k][i]
  if (first && lane < a.K) pv = a.prev[(size_t)lane * a.n_max + it.i];
  // the branch's MT-1 history samples (first chunks): with 8 outputs per lane
  // loaded before the z-pass, which then hides their latency; with 16 the
  // extra live registers across the z-pass cost more than that, so after it
  auto head = [&](int k) {
    float2 hx = make_float2(0.f, 0.f);
    const int f = __shfl_sync(0xffffffffu, pv, k);
    if (lane < MT - 1) {
      if (short_block) hx = hist_sample(a, pl, it.i, k, lane);
      else
        hx = f >= 0 ? reinterpret_cast<const float2*>(slot_at(a.data, pl.slot_data0, (uint32_t)f))
                          [a.L - (MT - 1) + lane]
                    : a.hist[((size_t)pl.parity_in * a.K + k) * (MT - 1) + lane];
    }
    return hx;
  };
  uint32_t rest = mask;
  while (rest) {
    const int k = __ffs(rest) - 1;
    rest &= rest - 1;
    const int q = (ok[k] - 1) >> 1;
    if constexpr (R == 8) {
      float2 hx = make_float2(0.f, 0.f);
      if (first) hx = head(k);
      zpass_w<R>(xs, zw, lane, q);
      if (first && lane < MT - 1) zstore(zw, lane, R, hx, upow(fmaf(hx.x, hx.x, hx.y * hx.y), q));
    } else {
      zpass_w<R>(xs, zw, lane, q);
      if (first) {
        const float2 hx = head(k);
        if (lane < MT - 1) zstore(zw, lane, R, hx, upow(fmaf(hx.x, hx.x, hx.y * hx.y), q));
      }
    }
    __syncwarp();
    fir_w<R, MT>(P, Q, zw, lane, hw + k * MT);
    __syncwarp();
  }
  float2 y[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float2 p = unpack_b64(P[r]), q = unpack_b64(Q[r]);
    y[r] = make_float2(p.x - q.y, p.y + q.x);
  }
  store_w<R>(yb, it.len, lane, y);
}

constexpr int kMaxGroup = 1024;

// `order` (may be null: identity) lists the group's actors in the order their
// items are laid out; actors of equal padded tap count are kept together, so
// that the warps of an SM, which work on neighbouring items, run the same
// code at the same time.
template <int R, int MTMAX>
__device__ inline void dpd_body_dev(const DpdArgs* __restrict__ args, const uint16_t* __restrict__ order,
                                    int G, Grid grid, float4* smem_raw) {
  using S = WarpSmem<R, MTMAX>;
  __shared__ uint64_t sw[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  constexpr uint32_t WI = 32 * R;
  uint64_t* s_off = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t carry = 0;
  for (int base = 0; base < G; base += blockDim.x) {
    const int j = base + threadIdx.x;
    uint64_t items = 0;
    if (j < G) {
      const DpdArgs& a = args[order ? order[j] : j];
      items = a.plan->n * ((a.L + WI - 1) / WI);
    }
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan_u64(items, sw, &tot);
    if (j < G) s_off[j] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) s_off[G] = carry;
  uint16_t* s_ord = reinterpret_cast<uint16_t*>(s_off + G + 1);
  for (int j = threadIdx.x; j < G; j += blockDim.x) s_ord[j] = order ? order[j] : (uint16_t)j;
  __syncthreads();
  const uint64_t total = carry;
  uint8_t* wb = reinterpret_cast<uint8_t*>(smem_raw) + dpd_body_off_bytes(G) + (size_t)wid * S::bytes;
  float2* xw = reinterpret_cast<float2*>(wb);
  float2* zw = reinterpret_cast<float2*>(wb + S::x_bytes);
  ulonglong2* hw = reinterpret_cast<ulonglong2*>(wb + S::x_bytes + S::z_bytes);
  uint32_t* mw = reinterpret_cast<uint32_t*>(wb + S::x_bytes + S::z_bytes + S::h_bytes);
  // Items are dealt to warps in runs of kRun consecutive items (a warp keeps
  // its actor's taps for a run): run r of global warp gw holds items
  // (r * NW + gw) * kRun .. + kRun - 1.  Runs of 4 when there are at least
  // 4 items per warp; a smaller step takes shorter runs, so that its items
  // spread over more warps instead of queueing behind one another.
  const uint64_t NW = (uint64_t)grid.n * nwarp;
  const int lg_run = total >= 4 * NW ? 2 : (total >= 2 * NW ? 1 : 0);      // kRun = 1 << lg_run
  const uint64_t gw = (uint64_t)wid * grid.n + grid.b;
  auto item_of = [&](uint64_t k) {
    return (((k >> lg_run) * NW + gw) << lg_run) + (k & ((1u << lg_run) - 1u));
  };
  uint64_t k = 0;
  int taps_of = -1;                                  // actor whose taps are in hw
  LocHint hint;
  WItem cur = locate_w(args, s_off, s_ord, G, item_of(0), total, WI, hint);
  if (cur.g >= 0) prefetch_w(args[cur.g], cur, xw, mw, WI, lane);
  cp_async_commit();
  int buf = 0;
  while (cur.g >= 0) {
    const DpdArgs& a = args[cur.g];
    if (cur.g != taps_of) {
      // taps {hx, hy} of every branch, then the branch orders, by asynchronous
      // copies waited for together with this item's x window
      for (int e = lane; e < a.K * a.MT; e += 32) cp_async16(hw + e, a.h + e);
      if (lane < a.K) {
        const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(
            reinterpret_cast<int32_t*>(hw + a.K * a.MT) + lane));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(a.orders + lane) : "memory");
      }
      taps_of = cur.g;
    }
    cp_async_commit();
    WItem nxt = locate_w(args, s_off, s_ord, G, item_of(k + 1), total, WI, hint);
    if (nxt.g >= 0) prefetch_w(args[nxt.g], nxt, xw + (buf ^ 1) * S::XW, mw + (buf ^ 1), WI, lane);
    cp_async_commit();
    cp_async_wait1();                                  // all but the next item's window
    __syncwarp();
    const float2* xs = xw + buf * S::XW + cur.shift;
    const uint32_t mask = mw[buf];
    if (mask == 0) {
      float2* yb = reinterpret_cast<float2*>(const_cast<uint8_t*>(slot_at(a.out, a.plan->slot_out0, cur.i))) +
                   cur.t0;
      float2 y[R];
#pragma unroll
      for (int r = 0; r < R; ++r) y[r] = make_float2(0.f, 0.f);
      store_w<R>(yb, cur.len, lane, y);
    } else {
      switch (a.MT) {
#define DPD_CASE(MTV) \
        case MTV: if constexpr (MTV <= MTMAX) dpd_item_w<R, MTV>(a, cur, mask, xs, zw, hw, lane); break;
        DPD_MT_CASES(DPD_CASE)
#undef DPD_CASE
        default: break;
      }
    }
    __syncwarp();
    cur = nxt;
    ++k;
    buf ^= 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // the histories for the next step, one CTA per actor counted from the last
  // CTA (the first CTAs take the first items, so a small step leaves these idle)
  for (int j = (int)(grid.n - 1 - grid.b); j < G; j += (int)grid.n) dpd_hist_dev(args[j]);
}

}  // namespace dfg
