// Device-side phases of the copy actor (shared by the per-phase kernels and
// the persistent step kernel).
//
// Copy actor (a static actor in the sense of Sec. 2.2): each firing consumes
// r_in tokens from its input and writes the same bytes, re-cut into r_out
// tokens, to every output.  Its plan is one thread: the number of firings is
// the largest n with n*r_in tokens present and n*r_out free slots on every
// output.  The plan commits the counters immediately; the body then moves the
// bytes of the n firings, wrapping around both rings.
#pragma once
#include "common.cuh"

namespace dfg {

__device__ inline void copy_plan_dev(const CopyArgs& a) {
  uint64_t* ctr = a.ctr;
  uint64_t rd = *rd_ptr(ctr, a.in.id), wr_in = *wr_ptr(ctr, a.in.id);
  uint64_t n = (wr_in - rd) / a.in.rate;
  for (int p = 0; p < a.n_out; ++p) {
    const ChanDesc& o = a.out[p];
    uint64_t occ = *wr_ptr(ctr, o.id) - *rd_ptr(ctr, o.id);
    uint64_t f = (o.cap - occ) / o.rate;
    n = f < n ? f : n;
  }
  a.plan->n = n;
  a.plan->rd0 = rd;
  *rd_ptr(ctr, a.in.id) = rd + n * a.in.rate;
  for (int p = 0; p < a.n_out; ++p) {
    uint64_t w = *wr_ptr(ctr, a.out[p].id);
    a.plan->wr0[p] = w;
    *wr_ptr(ctr, a.out[p].id) = w + n * a.out[p].rate;
  }
  atomicAdd(&a.eng->fired_total, (unsigned long long)n);
}

template <typename U>
__device__ inline void copy_units(const CopyArgs& a, const CopyPlan& pl, Grid g) {
  const uint64_t unit = sizeof(U);
  const uint64_t bytes = pl.n * a.in.rate * a.in.tok;
  const uint64_t n_units = bytes / unit;
  const uint64_t in_ring = a.in.cap * a.in.tok;
  const uint64_t in_off = (pl.rd0 % a.in.cap) * a.in.tok;
  const uint64_t stride = (uint64_t)g.n * blockDim.x;
  for (int p = 0; p < a.n_out; ++p) {
    const ChanDesc& o = a.out[p];
    const uint64_t out_ring = o.cap * o.tok;
    const uint64_t out_off = ((pl.wr0[p] - o.wshift) % o.cap) * o.tok;
    for (uint64_t u = g.b * (uint64_t)blockDim.x + threadIdx.x; u < n_units; u += stride) {
      uint64_t b = u * unit;
      uint64_t si = in_off + b;
      if (si >= in_ring) si -= in_ring;
      uint64_t di = out_off + b;
      if (di >= out_ring) di -= out_ring;
      *reinterpret_cast<U*>(o.ring + di) = *reinterpret_cast<const U*>(a.in.ring + si);
    }
  }
}

__device__ inline void copy_body_dev(const CopyArgs& a, Grid g) {
  const CopyPlan pl = *a.plan;
  if (pl.n == 0) return;
  if (a.unit == 16) copy_units<uint4>(a, pl, g);
  else if (a.unit == 4) copy_units<uint32_t>(a, pl, g);
  else copy_units<uint8_t>(a, pl, g);
}

// Spill of a delay channel in the paper's layout (Fig. 2): every CTA of the
// grid copies its share of the token in slot cap to slot 0.
__device__ inline void spill_dev(const SpillArgs& a, Grid g) {
  // tokens w0 .. w1-1 were written (w0 >= 1: the delay token is token 0)
  const uint64_t w1 = a.ctr[2 * a.id], w0 = *a.wr_before;
  if ((w1 - 1) / a.cap == (w0 - 1) / a.cap) return;
  const uint8_t* src = a.ring + a.cap * a.tok;
  const uint64_t stride = (uint64_t)g.n * blockDim.x;
  const uint64_t first = g.b * (uint64_t)blockDim.x + threadIdx.x;
  if (a.unit == 16) {
    for (uint64_t u = first; u < a.tok / 16; u += stride)
      reinterpret_cast<uint4*>(a.ring)[u] = reinterpret_cast<const uint4*>(src)[u];
  } else if (a.unit == 4) {
    for (uint64_t u = first; u < a.tok / 4; u += stride)
      reinterpret_cast<uint32_t*>(a.ring)[u] = reinterpret_cast<const uint32_t*>(src)[u];
  } else {
    for (uint64_t u = first; u < a.tok; u += stride) a.ring[u] = src[u];
  }
}

}  // namespace dfg
