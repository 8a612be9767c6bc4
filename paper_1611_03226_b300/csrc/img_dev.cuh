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
//                     shared memory by 16-byte asynchronous copies, the next
//                     band's while the current one is computed.
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
    a.plan->slot_in[i] = rd[i] % a.in[i].cap;
    *rd_ptr(ctr, a.in[i].id) = rd[i] + n * r;
  }
  for (int p = 0; p < a.n_out; ++p) {
    const uint64_t w = *wr_ptr(ctr, a.out[p].id);
    a.plan->wr0[p] = w;
    a.plan->slot_out[p] = (w - a.out[p].wshift) % a.out[p].cap;
    *wr_ptr(ctr, a.out[p].id) = w + n * r;
  }
  atomicAdd(&a.eng->fired_total, (unsigned long long)n);
}

// Frame f of this step's window of a channel whose first frame is in ring
// slot slot0 (f < capacity: a step never moves more frames than a ring holds).
__device__ __forceinline__ uint8_t* img_frame(const ChanDesc& c, uint64_t slot0, uint64_t f) {
  uint64_t s = slot0 + f;
  if (s >= c.cap) s -= c.cap;
  return c.ring + s * c.tok;
}

// q = it / d, r = it % d, with 32-bit arithmetic whenever it fits.
__device__ __forceinline__ void div_item(uint64_t it, uint32_t d, uint64_t& q, uint32_t& r) {
  if (it <= 0xffffffffull) {
    const uint32_t i = (uint32_t)it, qq = i / d;
    q = qq;
    r = i - qq * d;
  } else {
    q = it / d;
    r = (uint32_t)(it - q * d);
  }
}

// Median of five, per 16-bit lane, with the 3-input min/max instructions:
// med3(e, max(min(a,b), min(c,d)), min(max(a,b), max(c,d))).
__device__ __forceinline__ uint32_t med5_u16x2(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
  const uint32_t f = __vimax3_u16x2(__vimin3_u16x2(a, b, b), __vimin3_u16x2(c, d, d), 0u);
  const uint32_t g = __vimin3_u16x2(__vimax3_u16x2(a, b, 0u), __vimax3_u16x2(c, d, 0u),
                                    __vimax3_u16x2(c, d, 0u));
  return __vimax3_u16x2(__vimin3_u16x2(e, f, f), __vimin3_u16x2(e, g, g), __vimin3_u16x2(f, g, g));
}

// True when every byte of w is 0x00 or 0xff (bits 1..7 of each byte equal
// its bits 0..6).
__device__ __forceinline__ bool bytes_binary(uint32_t w) { return ((w ^ (w << 1)) & 0xfefefefeu) == 0; }

// Bitwise majority of five words (at least 3 of 5 bits set): for bytes that
// are 0x00 or 0xff this is the median of five.  With k = the count among c, d,
// e: a and b both set need k >= 1, one of them k >= 2, none k = 3 (and k = 3
// suffices alone); every term is one 3-input logic operation.
__device__ __forceinline__ uint32_t maj5(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
  const uint32_t any3 = c | d | e, two3 = (c & d) | (c & e) | (d & e), all3 = c & d & e;
  return (a & b & any3) | ((a | b) & two3) | all3;
}

// Median of five per byte: even and odd bytes in 16-bit lanes.
__device__ __forceinline__ uint32_t med5_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
  const uint32_t m = 0x00ff00ffu;
  const uint32_t lo = med5_u16x2(a & m, b & m, c & m, d & m, e & m);
  const uint32_t hi = med5_u16x2((a >> 8) & m, (b >> 8) & m, (c >> 8) & m, (d >> 8) & m, (e >> 8) & m);
  return lo | (hi << 8);
}

__device__ __forceinline__ uint4 thres4(uint4 x, uint4 y, uint32_t thr4) {
  return make_uint4(__vcmpgtu4(__vabsdiffu4(x.x, y.x), thr4), __vcmpgtu4(__vabsdiffu4(x.y, y.y), thr4),
                    __vcmpgtu4(__vabsdiffu4(x.z, y.z), thr4), __vcmpgtu4(__vabsdiffu4(x.w, y.w), thr4));
}

constexpr int kThresChunk = 4;     // frames per item when the previous frames are shared

// Thres when in[1] carries in[0]'s stream one token later: an item walks
// kThresChunk consecutive frames of one vector block, reading each current
// frame once and keeping it as the next frame's previous one; only the
// first frame of the chunk takes its previous frame from the other input
// (frame 0 of the window: the delay channel's own token).
__device__ inline void thres_dedup(const ImgArgs& a, const ImgPlan& pl, Grid g) {
  const uint64_t frames = pl.n * a.in[0].rate;
  const uint32_t vpf = (uint32_t)((uint64_t)a.W * a.H / 16);
  const uint32_t per_item = 4 * blockDim.x;
  const uint32_t ipf = (vpf + per_item - 1) / per_item;
  const uint64_t items = (frames + kThresChunk - 1) / kThresChunk * ipf;
  const uint32_t thr4 = 0x01010101u * (uint32_t)a.thr;
  for (uint64_t it = g.b; it < items; it += g.n) {
    uint64_t ch;
    uint32_t ci;
    div_item(it, ipf, ch, ci);
    const uint64_t j0 = ch * kThresChunk;
    const int nj = (int)min((uint64_t)kThresChunk, frames - j0);
    const uint32_t v0 = ci * per_item + threadIdx.x;
    const uint4* p = reinterpret_cast<const uint4*>(
        j0 == 0 ? img_frame(a.in[1], pl.slot_in[1], 0) : img_frame(a.in[0], pl.slot_in[0], j0 - 1));
    uint4 y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (v0 + k * blockDim.x < vpf) y[k] = p[v0 + k * blockDim.x];
    for (int j = 0; j < nj; ++j) {
      const uint4* c = reinterpret_cast<const uint4*>(img_frame(a.in[0], pl.slot_in[0], j0 + j));
      uint4* o = reinterpret_cast<uint4*>(img_frame(a.out[0], pl.slot_out[0], j0 + j));
      uint4 x[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (v0 + k * blockDim.x < vpf) x[k] = c[v0 + k * blockDim.x];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (v0 + k * blockDim.x < vpf) {
          o[v0 + k * blockDim.x] = thres4(x[k], y[k], thr4);
          y[k] = x[k];
        }
    }
  }
}

// Thres over whole frames: 255 where |cur - prev| > thr.
__device__ inline void thres_body(const ImgArgs& a, const ImgPlan& pl, Grid g) {
  if (a.dedup) {
    thres_dedup(a, pl, g);
    return;
  }
  const uint64_t frames = pl.n * a.in[0].rate;
  const uint32_t vpf = (uint32_t)((uint64_t)a.W * a.H / 16);        // 16-byte vectors per frame
  const uint32_t per_item = 4 * kImgThreads;
  const uint32_t ipf = (vpf + per_item - 1) / per_item;             // items per frame
  const uint64_t items = frames * ipf;
  const uint32_t thr4 = 0x01010101u * (uint32_t)a.thr;
  for (uint64_t it = g.b; it < items; it += g.n) {
    uint64_t f;
    uint32_t ci;
    div_item(it, ipf, f, ci);
    const uint32_t v0 = ci * per_item;
    const uint4* c = reinterpret_cast<const uint4*>(img_frame(a.in[0], pl.slot_in[0], f));
    const uint4* p = reinterpret_cast<const uint4*>(img_frame(a.in[1], pl.slot_in[1], f));
    uint4* o = reinterpret_cast<uint4*>(img_frame(a.out[0], pl.slot_out[0], f));
    // 4 vectors per thread, all loads issued before the first use
    uint4 x[4], y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t v = v0 + threadIdx.x + k * blockDim.x;
      if (v < vpf) {
        x[k] = c[v];
        y[k] = p[v];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t v = v0 + threadIdx.x + k * blockDim.x;
      if (v < vpf) {
        uint4 m;
        m.x = __vcmpgtu4(__vabsdiffu4(x[k].x, y[k].x), thr4);
        m.y = __vcmpgtu4(__vabsdiffu4(x[k].y, y[k].y), thr4);
        m.z = __vcmpgtu4(__vabsdiffu4(x[k].z, y[k].z), thr4);
        m.w = __vcmpgtu4(__vabsdiffu4(x[k].w, y[k].w), thr4);
        o[v] = m;
      }
    }
  }
}

// Start copying input rows y0-2 .. y0+band+1 (those inside the frame) of
// one frame into s (row y at s + (y - y0 + 2) * W) with 16-byte asynchronous
// copies; the caller commits and waits.
__device__ __forceinline__ void stage_rows(const uint8_t* frame, uint8_t* s, int W, int H, int y0, int band) {
  const int ya = max(y0 - 2, 0), yb = min(y0 + band + 2, H);
  const int vpr = W / 16;
  const int nv = (yb - ya) * vpr;
  const uint8_t* src = frame + (size_t)ya * W;
  uint8_t* dst = s + (size_t)(ya - y0 + 2) * W;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + 16 * v));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + 16 * v) : "memory");
  }
}
__device__ __forceinline__ void img_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void img_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// A thread's walk over the 16-pixel units of W-pixel rows: unit e = tid +
// k * blockDim.x of a row range is (row e / q, column e % q), q = W / 16.
// The start and the stride are fixed per thread, so they are computed once.
struct UnitMap {
  int row0, col0, drow, dcol, q;
};
__device__ __forceinline__ UnitMap unit_map(int W) {
  const int q = W / 16;
  return UnitMap{(int)threadIdx.x / q, (int)threadIdx.x % q, (int)blockDim.x / q, (int)blockDim.x % q, q};
}

// Calls f(y, x) for every row y in [ya, yb) and 16-pixel unit x = 0, 16, ..
// of the row, spread over the CTA's threads as the map says.
template <typename F>
__device__ __forceinline__ void for_units(const UnitMap& m, int ya, int yb, F&& f) {
  int y = ya + m.row0, c = m.col0;
  while (y < yb) {
    f(y, 16 * c);
    y += m.drow;
    c += m.dcol;
    if (c >= m.q) {
      c -= m.q;
      ++y;
    }
  }
}

// Band items (frame, band of img_band(W) rows) of this CTA with the input
// rows of the next item staged while the current one is computed (two
// buffers).  Items g.b, g.b + g.n, ..: (frame, band) advances by a fixed
// step, so it is carried along instead of divided out per item.
template <typename F>
__device__ __forceinline__ void for_band_items(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem,
                                               F&& compute) {
  const int W = a.W, H = a.H, band = img_band(W);
  const uint64_t frames = pl.n * a.in[0].rate;
  const uint32_t bands = (uint32_t)((H + band - 1) / band);
  const size_t sb = (size_t)(band + 4) * W;                        // one staging buffer
  uint64_t f;
  uint32_t b;
  div_item(g.b, bands, f, b);
  uint64_t fq;
  uint32_t fr;
  div_item(g.n, bands, fq, fr);
  auto next = [&](uint64_t& nf, uint32_t& nb) {
    nb += fr;
    nf += fq;
    if (nb >= bands) {
      nb -= bands;
      ++nf;
    }
  };
  __shared__ uint8_t* out_frames[kMaxPorts];
  int buf = 0;
  if (f < frames) stage_rows(img_frame(a.in[0], pl.slot_in[0], f), smem, W, H, (int)b * band, band);
  img_commit();
  while (f < frames) {
    uint64_t f1 = f;
    uint32_t b1 = b;
    next(f1, b1);
    if (f1 < frames) stage_rows(img_frame(a.in[0], pl.slot_in[0], f1), smem + (buf ^ 1) * sb, W, H, (int)b1 * band, band);
    img_commit();
    const int y0 = (int)b * band;
    // this item's output frames, one per port
    if (threadIdx.x < a.n_out) {
      const int p = threadIdx.x;
      out_frames[p] = img_frame(a.out[p], pl.slot_out[p], f);
    }
    img_wait_prev();
    __syncthreads();
    compute(y0, min(y0 + band, H), smem + buf * sb, out_frames);
    __syncthreads();
    buf ^= 1;
    f = f1;
    b = b1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Weighted vertical sum (1, 4, 6, 4, 1) of five rows' 4-pixel words: pixels
// 0 and 2 in the 16-bit lanes of lo, pixels 1 and 3 in those of hi (<= 16 * 255).
__device__ __forceinline__ void vsum5(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e,
                                      uint32_t& lo, uint32_t& hi) {
  lo = __byte_perm(a, 0, 0x4240) + __byte_perm(e, 0, 0x4240) +
       4u * (__byte_perm(b, 0, 0x4240) + __byte_perm(d, 0, 0x4240)) + 6u * __byte_perm(c, 0, 0x4240);
  hi = __byte_perm(a, 0, 0x4341) + __byte_perm(e, 0, 0x4341) +
       4u * (__byte_perm(b, 0, 0x4341) + __byte_perm(d, 0, 0x4341)) + 6u * __byte_perm(c, 0, 0x4341);
}

// Horizontal pass of 4 pixels from the vertical sums v[x-2] .. v[x+5] as four
// u16 pairs: pairs (v_i, v_{i+2}) for the even pixels x, x+2 and the odd
// pixels x+1, x+3; each 16-bit lane of the weighted sum stays below 65536.
__device__ __forceinline__ uint32_t hsum5(uint32_t w01, uint32_t w23, uint32_t w45, uint32_t w67) {
  const uint32_t s02 = __byte_perm(w01, w23, 0x5410), s13 = __byte_perm(w01, w23, 0x7632);
  const uint32_t s24 = __byte_perm(w23, w45, 0x5410), s35 = __byte_perm(w23, w45, 0x7632);
  const uint32_t s46 = __byte_perm(w45, w67, 0x5410), s57 = __byte_perm(w45, w67, 0x7632);
  const uint32_t he = s02 + 4 * s13 + 6 * s24 + 4 * s35 + s46 + 0x00800080u;
  const uint32_t ho = s13 + 4 * s24 + 6 * s35 + 4 * s46 + s57 + 0x00800080u;
  return ((he >> 8) & 0x00ff00ffu) | (((ho >> 8) & 0x00ff00ffu) << 8);
}

// Vertical sums: u16 rows of kImgVPitch(W) elements, pixel x at index x + 8
// (16-byte aligned for x % 16 == 0), clamped columns -2, -1 at 6, 7 and W, W+1
// at W + 8, W + 9.
__host__ __device__ constexpr int kImgVPitch(int W) { return W + 16; }

// Gauss over bands of img_band(W) rows, 16 pixels per thread and pass.  Vertical
// sums of the 5 rows go to shared memory; the horizontal pass then weights 5
// neighbouring sums, adds 128 and shifts right by 8.
__device__ inline void gauss_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  uint16_t* v = reinterpret_cast<uint16_t*>(smem + 2 * (size_t)(img_band(W) + 4) * W);
  const int vw = kImgVPitch(W);
  const UnitMap um = unit_map(W);
  for_band_items(a, pl, g, smem, [&](int y0, int y1, const uint8_t* s, uint8_t* const* of) {
    // vertical pass over the band's filtered rows (2 <= y < H-2)
    const int fa = max(y0, 2), fb = min(y1, H - 2);
    for_units(um, fa, fb, [&](int yr, int x) {
      const uint8_t* col = s + (yr - y0) * W + x;                   // row yr-2
      const uint4 r0 = *reinterpret_cast<const uint4*>(col);
      const uint4 r1 = *reinterpret_cast<const uint4*>(col + W);
      const uint4 r2 = *reinterpret_cast<const uint4*>(col + 2 * W);
      const uint4 r3 = *reinterpret_cast<const uint4*>(col + 3 * W);
      const uint4 r4 = *reinterpret_cast<const uint4*>(col + 4 * W);
      uint32_t lo[4], hi[4];
      vsum5(r0.x, r1.x, r2.x, r3.x, r4.x, lo[0], hi[0]);
      vsum5(r0.y, r1.y, r2.y, r3.y, r4.y, lo[1], hi[1]);
      vsum5(r0.z, r1.z, r2.z, r3.z, r4.z, lo[2], hi[2]);
      vsum5(r0.w, r1.w, r2.w, r3.w, r4.w, lo[3], hi[3]);
      uint16_t* vr = v + (yr - y0) * vw + 8;
      const uint4 p0 = make_uint4(__byte_perm(lo[0], hi[0], 0x5410), __byte_perm(lo[0], hi[0], 0x7632),
                                  __byte_perm(lo[1], hi[1], 0x5410), __byte_perm(lo[1], hi[1], 0x7632));
      const uint4 p1 = make_uint4(__byte_perm(lo[2], hi[2], 0x5410), __byte_perm(lo[2], hi[2], 0x7632),
                                  __byte_perm(lo[3], hi[3], 0x5410), __byte_perm(lo[3], hi[3], 0x7632));
      *reinterpret_cast<uint4*>(vr + x) = p0;
      *reinterpret_cast<uint4*>(vr + x + 8) = p1;
      if (x == 0) vr[-1] = vr[-2] = (uint16_t)p0.x;                 // clamped columns -1, -2
      if (x + 16 == W) vr[W] = vr[W + 1] = (uint16_t)(p1.w >> 16);  // clamped columns W, W+1
    });
    __syncthreads();
    // horizontal pass and the unfiltered rows
    for_units(um, y0, y1, [&](int y, int x) {
      uint4 out;
      if (y < 2 || y >= H - 2) {
        out = *reinterpret_cast<const uint4*>(s + (y - y0 + 2) * W + x);
      } else {
        // v[x-2] .. v[x+17] as ten u16 pairs
        const uint16_t* vr = v + (y - y0) * vw + 8 + x;
        const uint32_t w1 = *reinterpret_cast<const uint32_t*>(vr - 2);
        const uint4 qa = *reinterpret_cast<const uint4*>(vr);
        const uint4 qb = *reinterpret_cast<const uint4*>(vr + 8);
        const uint32_t w10 = *reinterpret_cast<const uint32_t*>(vr + 16);
        out.x = hsum5(w1, qa.x, qa.y, qa.z);
        out.y = hsum5(qa.y, qa.z, qa.w, qb.x);
        out.z = hsum5(qa.w, qb.x, qb.y, qb.z);
        out.w = hsum5(qb.y, qb.z, qb.w, w10);
      }
      const size_t o = (size_t)y * W + x;
      for (int p = 0; p < a.n_out; ++p) *reinterpret_cast<uint4*>(of[p] + o) = out;
    });
  });
}

// Any byte of w neither 0x00 nor 0xff: a nonzero word.
__device__ __forceinline__ uint32_t nonbinary_bits(uint32_t w) { return (w ^ (w << 1)) & 0xfefefefeu; }

// Med over bands of img_band(W) rows, 16 pixels per thread.  When every input
// byte of the band and its halo rows is 0 or 255 (every motion map) the median
// is a bitwise majority; otherwise the bytewise min/max network runs.  The
// test is one vote per band, skipped when the input is known to be binary
// (its writer is Thres).
__device__ inline void med_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  const UnitMap um = unit_map(W);
  const bool known_binary = a.binary_in != 0;
  for_band_items(a, pl, g, smem, [&](int y0, int y1, const uint8_t* s, uint8_t* const* of) {
    bool binary = true;
    if (!known_binary) {
      uint32_t nb = 0;
      for_units(um, max(y0 - 1, 0), min(y1 + 1, H), [&](int y, int x) {
        const uint4 c = *reinterpret_cast<const uint4*>(s + (y - y0 + 2) * W + x);
        nb |= nonbinary_bits(c.x) | nonbinary_bits(c.y) | nonbinary_bits(c.z) | nonbinary_bits(c.w);
      });
      binary = __syncthreads_or(nb != 0) == 0;
    }
    for_units(um, y0, y1, [&](int y, int x) {
      const uint8_t* row = s + (y - y0 + 2) * W;
      const uint4 c = *reinterpret_cast<const uint4*>(row + x);
      uint4 out = c;
      if (y >= 1 && y < H - 1) {
        const uint4 up = *reinterpret_cast<const uint4*>(row - W + x);
        const uint4 dn = *reinterpret_cast<const uint4*>(row + W + x);
        const uint32_t pw = x > 0 ? *reinterpret_cast<const uint32_t*>(row + x - 4) : 0u;
        const uint32_t nw = x + 16 < W ? *reinterpret_cast<const uint32_t*>(row + x + 16) : 0u;
        const uint32_t cw[6] = {pw, c.x, c.y, c.z, c.w, nw};
        const uint32_t uw[4] = {up.x, up.y, up.z, up.w}, dw[4] = {dn.x, dn.y, dn.z, dn.w};
        uint32_t m[4];
        if (binary) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            m[j] = maj5(uw[j], dw[j], __funnelshift_l(cw[j], cw[j + 1], 8), __funnelshift_r(cw[j + 1], cw[j + 2], 8),
                        cw[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            m[j] = med5_bytes(uw[j], dw[j], __funnelshift_l(cw[j], cw[j + 1], 8),
                              __funnelshift_r(cw[j + 1], cw[j + 2], 8), cw[j + 1]);
        }
        out = make_uint4(m[0], m[1], m[2], m[3]);
        if (x == 0) out.x = (out.x & 0xffffff00u) | (c.x & 0xffu);                 // column 0 copied
        if (x + 16 == W) out.w = (out.w & 0x00ffffffu) | (c.w & 0xff000000u);      // column W-1 copied
      }
      const size_t o = (size_t)y * W + x;
      for (int p = 0; p < a.n_out; ++p) *reinterpret_cast<uint4*>(of[p] + o) = out;
    });
  });
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
