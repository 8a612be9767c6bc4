// Device-side phases of the bitmask-controlled dynamic actors (shared by the
// per-phase kernels and the persistent step kernel).
//
// Bitmask-controlled dynamic actors of the expanded predistorter network
// (Sec. 4.2: the Poly and Adder actors whose branch ports carry 0 or 1 token
// per firing, selected by the control token).
//
// Plan (one CTA): read the pending control tokens; for every regular port p an
// exclusive scan over the firings of its 0/1 activity gives rank[p][i]; firing
// i is enabled iff, on every port active in it, (rank + 1) * rate tokens are
// present (inputs) or free (outputs).  The enabled count n is the first index
// where some port fails (the scan is monotone, so this is the longest
// prefix); the counters are committed by the total activity of the prefix.
// Bodies: Poly writes |x|^(o_k-1) x of its input block to every active branch
// output; Adder sums the active branch inputs (ascending k; no active branch
// gives zeros).  Both are elementwise over blocks, one work item per
// (firing, port, tile).
#pragma once
#include "common.cuh"

namespace dfg {


__device__ inline uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t* sw, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sw[lane] = s;
  }
  __syncthreads();
  const uint32_t before = wid ? sw[wid - 1] : 0;
  *total = sw[nw - 1];
  __syncthreads();
  return before + x - v;
}

__device__ inline void dyn_plan_dev(const DynArgs& a) {
  __shared__ uint64_t s_base[kDynPorts], s_limit[kDynPorts];
  __shared__ uint64_t s_rdc;
  __shared__ unsigned long long s_n;
  __shared__ uint32_t sw[32];
  uint64_t* ctr = a.ctr;
  if (threadIdx.x == 0) {
    const uint64_t rdc = *rd_ptr(ctr, a.ctrl.id), wrc = *wr_ptr(ctr, a.ctrl.id);
    s_rdc = rdc;
    s_n = min(wrc - rdc, (uint64_t)a.n_max);
  }
  if (threadIdx.x < a.np) {
    const ChanDesc& c = a.port[threadIdx.x];
    const uint64_t wr = *wr_ptr(ctr, c.id), rd = *rd_ptr(ctr, c.id);
    s_base[threadIdx.x] = a.is_out[threadIdx.x] ? wr : rd;
    s_limit[threadIdx.x] = a.is_out[threadIdx.x] ? c.cap - (wr - rd) : wr - rd;
  }
  __syncthreads();
  const uint32_t n_ctrl = (uint32_t)s_n;
  for (uint32_t i = threadIdx.x; i < n_ctrl; i += blockDim.x)
    a.masks[i] = *reinterpret_cast<const uint32_t*>(slot_ptr(a.ctrl, s_rdc + i));
  __syncthreads();
  for (int p = 0; p < a.np; ++p) {
    const int bit = a.bit[p];
    const uint64_t rate = a.port[p].rate, limit = s_limit[p];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_ctrl; base += blockDim.x) {
      const uint32_t i = base + threadIdx.x;
      uint32_t act = 0;
      if (i < n_ctrl) act = bit < 0 ? 1u : (a.masks[i] >> bit) & 1u;
      uint32_t tot;
      const uint32_t ex = block_exclusive_scan_u32(act, sw, &tot);
      if (i < n_ctrl) {
        a.rank[(size_t)p * a.n_max + i] = carry + ex;
        if (act && (uint64_t)(carry + ex + 1) * rate > limit) atomicMin(&s_n, (unsigned long long)i);
      }
      carry += tot;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t n = (uint32_t)s_n;
    a.plan->n = n;
    *rd_ptr(ctr, a.ctrl.id) = s_rdc + n;
    atomicAdd(&a.eng->fired_total, (unsigned long long)n);
  }
  __syncthreads();
  const uint32_t n = (uint32_t)s_n;
  if (threadIdx.x < a.np) {
    const int p = threadIdx.x;
    // total activity of the first n firings = rank of firing n (or the full count)
    uint32_t used = 0;
    if (n > 0) {
      const uint32_t last = n - 1;
      const int bit = a.bit[p];
      const uint32_t act = bit < 0 ? 1u : (a.masks[last] >> bit) & 1u;
      used = a.rank[(size_t)p * a.n_max + last] + act;
    }
    a.plan->base[p] = s_base[p];
    const uint64_t moved = (uint64_t)used * a.port[p].rate;
    if (a.is_out[p]) *wr_ptr(ctr, a.port[p].id) = s_base[p] + moved;
    else *rd_ptr(ctr, a.port[p].id) = s_base[p] + moved;
  }
}

constexpr uint32_t kDynTile = 2048;

__device__ __forceinline__ float2 psi_q2(float2 x, int q) {
  const float u = fmaf(x.x, x.x, x.y * x.y);
  float p = 1.f;
  for (int i = 0; i < q; ++i) p *= u;
  return make_float2(p * x.x, p * x.y);
}

// Token of port p used by firing i (rate 1 ports).
__device__ __forceinline__ float2* port_token(const DynArgs& a, const DynPlanHdr& pl, int p, uint32_t i) {
  return reinterpret_cast<float2*>(slot_ptr(a.port[p], pl.base[p] + a.rank[(size_t)p * a.n_max + i]));
}

__device__ inline void poly_body_dev(const DynArgs& a, Grid g) {
  const DynPlanHdr* pl = a.plan;
  const uint64_t n = pl->n;
  const uint32_t nt = (a.L + kDynTile - 1) / kDynTile;
  const uint64_t items = n * a.K * nt;
  for (uint64_t it = g.b; it < items; it += g.n) {
    const uint32_t i = (uint32_t)(it / ((uint64_t)a.K * nt));
    const uint32_t rem = (uint32_t)(it % ((uint64_t)a.K * nt));
    const int k = (int)(rem / nt);
    const uint32_t t0 = (rem % nt) * kDynTile;
    if (!((a.masks[i] >> k) & 1u)) continue;
    const float2* x = port_token(a, *pl, 0, i);
    float2* z = port_token(a, *pl, 1 + k, i);
    const int q = (a.orders[k] - 1) >> 1;
    const uint32_t end = min(a.L, t0 + kDynTile);
    for (uint32_t s = t0 + threadIdx.x; s < end; s += blockDim.x) z[s] = psi_q2(x[s], q);
  }
}

__device__ inline void add_body_dev(const DynArgs& a, Grid g) {
  const DynPlanHdr* pl = a.plan;
  const uint64_t n = pl->n;
  const uint32_t nt = (a.L + kDynTile - 1) / kDynTile;
  const uint64_t items = n * nt;
  for (uint64_t it = g.b; it < items; it += g.n) {
    const uint32_t i = (uint32_t)(it / nt);
    const uint32_t t0 = (uint32_t)(it % nt) * kDynTile;
    const uint32_t mask = a.masks[i];
    float2* y = port_token(a, *pl, a.K, i);
    const uint32_t end = min(a.L, t0 + kDynTile);
    for (uint32_t s = t0 + threadIdx.x; s < end; s += blockDim.x) {
      float2 acc = make_float2(0.f, 0.f);
      for (int k = 0; k < a.K; ++k) {
        if ((mask >> k) & 1u) {
          const float2 v = port_token(a, *pl, k, i)[s];
          acc.x += v.x;
          acc.y += v.y;
        }
      }
      y[s] = acc;
    }
  }
}

}  // namespace dfg
