// Device-side phases of the image actors of the paper's own motion pipeline
// (Sec. 4.1): Gauss (5x5 Gaussian, two top and two bottom rows unfiltered),
// Thres (consecutive filtered frames, strict threshold, 255/0) and Med
// (5-pixel median), each a static actor whose every port carries r frames per
// firing.  Shared by the per-phase kernels and the persistent step kernel.
//
// plan  (one thread)  n = the largest number of firings with n*r frames on
//                     every input and n*r free slots on every output; the
//                     counters are committed at once (as for the copy actor).
// body  (any grid)    work items over the n*r frames of the step: Thres by
//                     16-byte vectors, Gauss and Med by bands of 16 output
//                     rows whose input rows (plus a 2-row halo) are staged in
//                     shared memory with 16-byte loads.
#pragma once
#include "common.cuh"

namespace dfg {

__device__ inline void img_plan_dev(const ImgArgs& a) {
  uint64_t* ctr = a.ctr;
  const uint64_t r = a.in[0].rate;
  uint64_t n = ~0ull;
  uint64_t rd[2] = {0, 0};
  for (int i = 0; i < a.n_in; ++i) {
    rd[i] = *rd_ptr(ctr, a.in[i].id);
    const uint64_t f = (*wr_ptr(ctr, a.in[i].id) - rd[i]) / r;
    n = f < n ? f : n;
  }
  for (int p = 0; p < a.n_out; ++p) {
    const ChanDesc& o = a.out[p];
    const uint64_t occ = *wr_ptr(ctr, o.id) - *rd_ptr(ctr, o.id);
    const uint64_t f = (o.cap - occ) / r;
    n = f < n ? f : n;
  }
  a.plan->n = n;
  for (int i = 0; i < a.n_in; ++i) {
    a.plan->rd0[i] = rd[i];
    *rd_ptr(ctr, a.in[i].id) = rd[i] + n * r;
  }
  for (int p = 0; p < a.n_out; ++p) {
    const uint64_t w = *wr_ptr(ctr, a.out[p].id);
    a.plan->wr0[p] = w;
    *wr_ptr(ctr, a.out[p].id) = w + n * r;
  }
  atomicAdd(&a.eng->fired_step, (unsigned long long)n);
  atomicAdd(&a.eng->fired_total, (unsigned long long)n);
}

// Frame f of this step's window of a channel.
__device__ __forceinline__ uint8_t* img_frame(const ChanDesc& c, uint64_t t0, uint64_t f) {
  return c.ring + ((t0 + f) % c.cap) * c.tok;
}

// Median of five bytewise (per byte lane): med3(e, max(min(a,b), min(c,d)), min(max(a,b), max(c,d))).
__device__ __forceinline__ uint32_t med5_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
  const uint32_t f = __vmaxu4(__vminu4(a, b), __vminu4(c, d));
  const uint32_t g = __vminu4(__vmaxu4(a, b), __vmaxu4(c, d));
  return __vmaxu4(__vminu4(e, f), __vminu4(__vmaxu4(e, f), g));
}

// Thres over whole frames: 255 where |cur - prev| > thr.
__device__ inline void thres_body(const ImgArgs& a, const ImgPlan& pl, Grid g) {
  const uint64_t frames = pl.n * a.in[0].rate;
  const uint32_t vpf = (uint32_t)((uint64_t)a.W * a.H / 16);        // 16-byte vectors per frame
  const uint32_t per_item = 4 * kImgThreads;
  const uint32_t ipf = (vpf + per_item - 1) / per_item;             // items per frame
  const uint64_t items = frames * ipf;
  const uint32_t thr4 = 0x01010101u * (uint32_t)a.thr;
  for (uint64_t it = g.b; it < items; it += g.n) {
    const uint64_t f = it / ipf;
    const uint32_t v0 = (uint32_t)(it - f * ipf) * per_item;
    const uint4* c = reinterpret_cast<const uint4*>(img_frame(a.in[0], pl.rd0[0], f));
    const uint4* p = reinterpret_cast<const uint4*>(img_frame(a.in[1], pl.rd0[1], f));
    uint4* o = reinterpret_cast<uint4*>(img_frame(a.out[0], pl.wr0[0], f));
    for (uint32_t v = v0 + threadIdx.x; v < min(vpf, v0 + per_item); v += blockDim.x) {
      const uint4 x = c[v], y = p[v];
      uint4 m;
      m.x = __vcmpgtu4(__vabsdiffu4(x.x, y.x), thr4);
      m.y = __vcmpgtu4(__vabsdiffu4(x.y, y.y), thr4);
      m.z = __vcmpgtu4(__vabsdiffu4(x.z, y.z), thr4);
      m.w = __vcmpgtu4(__vabsdiffu4(x.w, y.w), thr4);
      o[v] = m;
    }
  }
}

// Stage input rows y0-2 .. y0+kImgBand+1 (those inside the frame) of one
// frame into s (row y at s + (y - y0 + 2) * W).
__device__ __forceinline__ void stage_rows(const uint8_t* frame, uint8_t* s, int W, int H, int y0) {
  const int ya = max(y0 - 2, 0), yb = min(y0 + kImgBand + 2, H);
  const int vpr = W / 16;
  const int nv = (yb - ya) * vpr;
  const uint4* src = reinterpret_cast<const uint4*>(frame + (size_t)ya * W);
  uint4* dst = reinterpret_cast<uint4*>(s + (size_t)(ya - y0 + 2) * W);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = src[v];
}

// Gauss over bands of kImgBand rows.  Vertical sums of the 5 rows (weights
// 1, 4, 6, 4, 1) go to shared memory as u16 (<= 16 * 255) with the edge
// columns repeated twice on each side; the horizontal pass then weights 5
// neighbouring sums, adds 128 and shifts right by 8.
__device__ inline void gauss_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  const uint64_t frames = pl.n * a.in[0].rate;
  const int bands = (H + kImgBand - 1) / kImgBand;
  const uint64_t items = frames * bands;
  uint8_t* s = smem;                                                // (kImgBand + 4) rows
  uint16_t* v = reinterpret_cast<uint16_t*>(smem + (size_t)(kImgBand + 4) * W);   // 16-byte aligned (W % 16 == 0)
  const int vw = W + 4;                                             // u16 per vertical-sum row
  const int q = W / 4;                                              // 4-pixel groups per row
  for (uint64_t it = g.b; it < items; it += g.n) {
    const uint64_t f = it / bands;
    const int y0 = (int)(it - f * bands) * kImgBand;
    const int y1 = min(y0 + kImgBand, H);
    stage_rows(img_frame(a.in[0], pl.rd0[0], f), s, W, H, y0);
    __syncthreads();
    // vertical pass over the band's filtered rows (2 <= y < H-2)
    const int fa = max(y0, 2), fb = min(y1, H - 2);
    for (int e = threadIdx.x; e < (fb > fa ? (fb - fa) * q : 0); e += blockDim.x) {
      const int yr = fa + e / q, x = (e % q) * 4;
      uint32_t lo = 0, hi = 0;                                      // pixels x, x+2 / x+1, x+3 in 16-bit lanes
      const uint8_t* col = s + (size_t)(yr - y0) * W + x;           // row yr-2
#pragma unroll
      for (int dy = 0; dy < 5; ++dy) {
        const uint32_t w = *reinterpret_cast<const uint32_t*>(col + dy * W);
        const uint32_t k = dy == 2 ? 6u : (dy == 1 || dy == 3) ? 4u : 1u;
        lo += k * (w & 0x00ff00ffu);
        hi += k * ((w >> 8) & 0x00ff00ffu);
      }
      uint16_t* vr = v + (size_t)(yr - y0) * vw + 2;
      const uint32_t p01 = __byte_perm(lo, hi, 0x5410), p23 = __byte_perm(lo, hi, 0x7632);
      vr[x] = (uint16_t)p01;
      vr[x + 1] = (uint16_t)(p01 >> 16);
      vr[x + 2] = (uint16_t)p23;
      vr[x + 3] = (uint16_t)(p23 >> 16);
      if (x == 0) vr[-1] = vr[-2] = (uint16_t)p01;                  // clamped columns -1, -2
      if (x + 4 == W) vr[W] = vr[W + 1] = (uint16_t)(p23 >> 16);    // clamped columns W, W+1
    }
    __syncthreads();
    // horizontal pass and the unfiltered rows; 4 pixels per thread
    for (int e = threadIdx.x; e < (y1 - y0) * q; e += blockDim.x) {
      const int y = y0 + e / q, x = (e % q) * 4;
      uint32_t out;
      if (y < 2 || y >= H - 2) {
        out = *reinterpret_cast<const uint32_t*>(s + (size_t)(y - y0 + 2) * W + x);
      } else {
        const uint16_t* vr = v + (size_t)(y - y0) * vw + x;         // v[x-2] .. v[x+5]
        uint32_t t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = vr[i];
        out = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t h = t[j] + 4 * t[j + 1] + 6 * t[j + 2] + 4 * t[j + 3] + t[j + 4];
          out |= ((h + 128) >> 8) << (8 * j);
        }
      }
      for (int p = 0; p < a.n_out; ++p)
        *reinterpret_cast<uint32_t*>(img_frame(a.out[p], pl.wr0[p], f) + (size_t)y * W + x) = out;
    }
    __syncthreads();
  }
}

// Med over bands of kImgBand rows; 4 pixels per thread with bytewise min/max.
__device__ inline void med_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  const uint64_t frames = pl.n * a.in[0].rate;
  const int bands = (H + kImgBand - 1) / kImgBand;
  const uint64_t items = frames * bands;
  uint8_t* s = smem;
  const int q = W / 4;
  for (uint64_t it = g.b; it < items; it += g.n) {
    const uint64_t f = it / bands;
    const int y0 = (int)(it - f * bands) * kImgBand;
    const int y1 = min(y0 + kImgBand, H);
    stage_rows(img_frame(a.in[0], pl.rd0[0], f), s, W, H, y0);
    __syncthreads();
    for (int e = threadIdx.x; e < (y1 - y0) * q; e += blockDim.x) {
      const int y = y0 + e / q, x = (e % q) * 4;
      const uint8_t* row = s + (size_t)(y - y0 + 2) * W;
      const uint32_t c = *reinterpret_cast<const uint32_t*>(row + x);
      uint32_t out = c;
      if (y >= 1 && y < H - 1) {
        const uint32_t up = *reinterpret_cast<const uint32_t*>(row - W + x);
        const uint32_t dn = *reinterpret_cast<const uint32_t*>(row + W + x);
        const uint32_t pw = x >= 4 ? *reinterpret_cast<const uint32_t*>(row + x - 4) : 0u;
        const uint32_t nw = x + 4 < W ? *reinterpret_cast<const uint32_t*>(row + x + 4) : 0u;
        const uint32_t lf = __funnelshift_l(pw, c, 8);              // pixels x-1 .. x+2
        const uint32_t rt = __funnelshift_r(c, nw, 8);              // pixels x+1 .. x+4
        out = med5_bytes(up, dn, lf, rt, c);
        if (x == 0) out = (out & 0xffffff00u) | (c & 0xffu);        // column 0 copied
        if (x + 4 == W) out = (out & 0x00ffffffu) | (c & 0xff000000u);   // column W-1 copied
      }
      for (int p = 0; p < a.n_out; ++p)
        *reinterpret_cast<uint32_t*>(img_frame(a.out[p], pl.wr0[p], f) + (size_t)y * W + x) = out;
    }
    __syncthreads();
  }
}

__device__ inline void img_body_dev(const ImgArgs& a, Grid g, uint8_t* smem) {
  __shared__ ImgPlan s_pl;
  __syncthreads();
  if (threadIdx.x == 0) s_pl = *a.plan;
  __syncthreads();
  const ImgPlan& pl = s_pl;                  // read in place (wr0[] is indexed per port)
  if (pl.n == 0) return;
  if (a.kind == DF_THRES) thres_body(a, pl, g);
  else if (a.kind == DF_GAUSS5) gauss_body(a, pl, g, smem);
  else med_body(a, pl, g, smem);
}

}  // namespace dfg
