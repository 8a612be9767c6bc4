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

// ---------------------------------------------------- band staging ----
// The input rows of a band item (band rows plus a 2-row halo each side, those
// inside the frame) are contiguous in the frame, so one bulk asynchronous
// copy, issued by one thread and completing on an mbarrier, stages them.
__device__ __forceinline__ uint32_t img_smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ long long img_timer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool img_bar_done(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait until the phase of the given parity has completed, at most limit_ns.
__device__ __forceinline__ bool img_bar_wait(uint32_t bar, uint32_t parity, long long limit_ns) {
  if (img_bar_done(bar, parity)) return true;
  const long long t0 = img_timer_ns();
  while (!img_bar_done(bar, parity))
    if (img_timer_ns() - t0 > limit_ns) return false;
  return true;
}
// Thread 0: the rows of item (frame f, band starting at row y0) into buffer s
// (row y at s + (y - y0 + 2) * W), completing on bar.
__device__ __forceinline__ void img_stage(const uint8_t* frame, uint8_t* s, int W, int H, int y0, int band,
                                          uint32_t bar) {
  const int ya = max(y0 - 2, 0), yb = min(y0 + band + 2, H);
  const uint32_t bytes = (uint32_t)(yb - ya) * (uint32_t)W;        // a multiple of 16 (W is)
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   img_smem_addr(s + (size_t)(ya - y0 + 2) * W)),
               "l"(frame + (size_t)ya * W), "r"(bytes), "r"(bar)
               : "memory");
}

// The 16-pixel units of one band that a thread takes: units e = tid, tid +
// blockDim, .. of the band's band * q units (q = W / 16) are (row e / q,
// column 16 (e % q)); the first and the step are fixed per thread, so they
// are computed once and the walk steps instead of dividing.
struct BandUnits {
  int n;                       // units of this thread in a full band
  int dy0, c0;                 // first unit: row within the band, column / 16
  int drow, dcol, q;           // step between the thread's units
};
__device__ __forceinline__ BandUnits band_units(int W, int band) {
  const int q = W / 16, total = band * q, t = (int)threadIdx.x, nt = (int)blockDim.x;
  return BandUnits{t < total ? (total - t + nt - 1) / nt : 0, t / q, t % q, nt / q, nt % q, q};
}

// Band items (frame, band of img_band(W) rows) of this CTA, the rows of the
// next kImgBufs - 1 items staged while the current one is computed (a ring of
// kImgBufs buffers, one mbarrier each).  Items g.b, g.b + g.n, ..: (frame,
// band) advances by a fixed step, so it is carried along instead of divided
// out per item.  unit(y, x, row) returns the 16 output pixels of unit (y, x),
// row = its row y in the staging buffer; they are stored to every output
// frame.  Every wait is bounded: one that runs out records DF_ETIMEOUT, and
// thread 0 waits (bounded) for the copies still in flight before the CTA
// leaves.
template <typename F>
__device__ __forceinline__ void for_band_items(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem,
                                               F&& unit) {
  constexpr int NB = kImgBufs;
  const int W = a.W, H = a.H, band = img_band(W);
  const uint64_t frames = pl.n * a.in[0].rate;
  const uint32_t bands = (uint32_t)((H + band - 1) / band);
  const size_t sb = (size_t)(band + 4) * W;                        // one staging buffer
  const long long limit = a.wait_limit_ns;
  __shared__ __align__(8) unsigned long long s_bar[NB];
  __shared__ uint8_t* out_frames[kMaxPorts];
  const uint32_t bar0 = img_smem_addr(&s_bar[0]);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NB; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * i) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const BandUnits bu = band_units(W, band);
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
  uint64_t f, fa;                      // the item computed next; the next item to stage
  uint32_t b, ba;
  div_item(g.b, bands, f, b);
  fa = f;
  ba = b;
  uint32_t phase = 0;                  // bit i: parity of buffer i's next phase
  uint32_t pending = 0;                // bit i: a copy into buffer i not yet waited for
  for (int i = 0; i < NB - 1; ++i) {
    if (fa < frames) {
      if (threadIdx.x == 0)
        img_stage(img_frame(a.in[0], pl.slot_in[0], fa), smem + i * sb, W, H, (int)ba * band, band, bar0 + 8 * i);
      pending |= 1u << i;
    }
    next(fa, ba);
  }
  int buf = 0;
  bool ok = true;
  while (f < frames) {
    // the buffer computed last (released by the barrier that ended it) takes
    // the item NB - 1 ahead
    const int sa = buf == 0 ? NB - 1 : buf - 1;
    if (fa < frames) {
      if (threadIdx.x == 0)
        img_stage(img_frame(a.in[0], pl.slot_in[0], fa), smem + sa * sb, W, H, (int)ba * band, band,
                  bar0 + 8 * sa);
      pending |= 1u << sa;
    }
    next(fa, ba);
    if (threadIdx.x < a.n_out) out_frames[threadIdx.x] = img_frame(a.out[threadIdx.x], pl.slot_out[threadIdx.x], f);
    const bool arrived = img_bar_wait(bar0 + 8 * buf, (phase >> buf) & 1u, limit);
    if (!__syncthreads_and(arrived)) {
      ok = false;
      break;
    }
    phase ^= 1u << buf;
    pending &= ~(1u << buf);
    const int y0 = (int)b * band, y1 = min(y0 + band, H);
    const uint8_t* s = smem + buf * sb;
    uint8_t* o0 = out_frames[0] + (size_t)y0 * W;
    uint8_t* o1 = a.n_out > 1 ? out_frames[1] + (size_t)y0 * W : nullptr;
    int dy = bu.dy0, c = bu.c0;
    for (int k = 0; k < bu.n; ++k) {
      if (y0 + dy < y1) {
        const int x = 16 * c;
        const int o = dy * W + x;                      // within the band's rows
        const uint4 out = unit(y0 + dy, x, s + 2 * W + o);
        *reinterpret_cast<uint4*>(o0 + o) = out;
        if (o1) *reinterpret_cast<uint4*>(o1 + o) = out;
        for (int p = 2; p < a.n_out; ++p) *reinterpret_cast<uint4*>(out_frames[p] + (size_t)y0 * W + o) = out;
      }
      dy += bu.drow;
      c += bu.dcol;
      if (c >= bu.q) {
        c -= bu.q;
        ++dy;
      }
    }
    __syncthreads();
    buf = buf == NB - 1 ? 0 : buf + 1;
    next(f, b);
  }
  if (!ok && threadIdx.x == 0) {
    set_status(a.eng, DF_ETIMEOUT, kWhereImgStage);
    for (int i = 0; i < NB; ++i)
      if (pending & (1u << i)) img_bar_wait(bar0 + 8 * i, (phase >> i) & 1u, limit);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the barriers may be initialised again by a later call (persistent kernel)
    for (int i = 0; i < NB; ++i) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0 + 8 * i) : "memory");
  }
  __syncthreads();
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

// Horizontal (1, 4, 6, 4, 1) of 4 pixels x .. x+3 from 16-bit pairs of
// vertical sums: A = (v[x-2], v[x]), B = (v[x-1], v[x+1]), lo = (v[x], v[x+2]),
// hi = (v[x+1], v[x+3]), E = (v[x+2], v[x+4]), F = (v[x+3], v[x+5]); + 128, >> 8
// (each 16-bit lane stays below 65536), the four result bytes picked out by
// one byte permute.
__device__ __forceinline__ uint32_t hsum5p(uint32_t A, uint32_t B, uint32_t lo, uint32_t hi, uint32_t E,
                                           uint32_t F) {
  const uint32_t he = A + 4u * (B + hi) + 6u * lo + E + 0x00800080u;  // pixels x, x+2
  const uint32_t ho = B + 4u * (lo + E) + 6u * hi + F + 0x00800080u;  // pixels x+1, x+3
  return __byte_perm(he, ho, 0x7351);
}

// Gauss over bands of img_band(W) rows, 16 pixels per thread: from the staged
// rows y-2 .. y+2, the unit's 16 pixels and one word on each side give the
// vertical sums in registers, then the horizontal pass; one pass per band, no
// second barrier.  Columns -2, -1 and W, W+1 repeat columns 0 and W-1; rows
// 0, 1, H-2, H-1 are copied.
__device__ inline void gauss_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  for_band_items(a, pl, g, smem, [&](int y, int x, const uint8_t* row) -> uint4 {
      uint4 out;
      if (y < 2 || y >= H - 2) {
        out = *reinterpret_cast<const uint4*>(row);
      } else {
        // rows y-2 .. y+2: the unit's 16 pixels, and pixels x-2, x-1, x+16,
        // x+17 gathered into one word per row
        uint4 m[5];
        uint32_t e[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          const uint8_t* ri = row + (i - 2) * W;
          m[i] = *reinterpret_cast<const uint4*>(ri);
          const uint32_t l = x > 0 ? *reinterpret_cast<const uint32_t*>(ri - 4) : 0u;
          const uint32_t r = x + 16 < W ? *reinterpret_cast<const uint32_t*>(ri + 16) : 0u;
          e[i] = __byte_perm(l, r, 0x5432);
        }
        // vertical sums: lo[w] = (v[4w], v[4w+2]), hi[w] = (v[4w+1], v[4w+3]);
        // le = (v[-2], v[16]), he_ = (v[-1], v[17])
        uint32_t lo[4], hi[4], le, he_;
        vsum5(m[0].x, m[1].x, m[2].x, m[3].x, m[4].x, lo[0], hi[0]);
        vsum5(m[0].y, m[1].y, m[2].y, m[3].y, m[4].y, lo[1], hi[1]);
        vsum5(m[0].z, m[1].z, m[2].z, m[3].z, m[4].z, lo[2], hi[2]);
        vsum5(m[0].w, m[1].w, m[2].w, m[3].w, m[4].w, lo[3], hi[3]);
        vsum5(e[0], e[1], e[2], e[3], e[4], le, he_);
        if (x == 0) {                                                       // v[-2] = v[-1] = v[0]
          le = (le & 0xffff0000u) | (lo[0] & 0xffffu);
          he_ = (he_ & 0xffff0000u) | (lo[0] & 0xffffu);
        }
        if (x + 16 == W) {                                                  // v[16] = v[17] = v[15]
          le = (le & 0xffffu) | (hi[3] & 0xffff0000u);
          he_ = (he_ & 0xffffu) | (hi[3] & 0xffff0000u);
        }
        // pairs (v[4w-2], v[4w]) and (v[4w-1], v[4w+1]), w = 0 .. 4
        uint32_t A[5], B[5];
        A[0] = __byte_perm(le, lo[0], 0x5410);
        B[0] = __byte_perm(he_, hi[0], 0x5410);
#pragma unroll
        for (int w = 1; w < 4; ++w) {
          A[w] = __byte_perm(lo[w - 1], lo[w], 0x5432);
          B[w] = __byte_perm(hi[w - 1], hi[w], 0x5432);
        }
        A[4] = __byte_perm(lo[3], le, 0x7632);
        B[4] = __byte_perm(hi[3], he_, 0x7632);
        out = make_uint4(hsum5p(A[0], B[0], lo[0], hi[0], A[1], B[1]), hsum5p(A[1], B[1], lo[1], hi[1], A[2], B[2]),
                         hsum5p(A[2], B[2], lo[2], hi[2], A[3], B[3]), hsum5p(A[3], B[3], lo[3], hi[3], A[4], B[4]));
      }
      return out;
  });
}

// Any byte of w neither 0x00 nor 0xff: a nonzero word.
__device__ __forceinline__ uint32_t nonbinary_bits(uint32_t w) { return (w ^ (w << 1)) & 0xfefefefeu; }

// Med over bands of img_band(W) rows, 16 pixels per thread.  When the input
// is known to be binary (its writer is Thres and its initial tokens are 0 or
// 255), or every word a unit reads is, the median of five is a bitwise
// majority; otherwise the bytewise min/max network runs.  Rows 0 and H-1 and
// columns 0 and W-1 are copied.
__device__ inline void med_body(const ImgArgs& a, const ImgPlan& pl, Grid g, uint8_t* smem) {
  const int W = a.W, H = a.H;
  const bool known_binary = a.binary_in != 0;
  for_band_items(a, pl, g, smem, [&](int y, int x, const uint8_t* row) -> uint4 {
    const uint4 c = *reinterpret_cast<const uint4*>(row);
    if (y < 1 || y >= H - 1) return c;
    const uint4 up = *reinterpret_cast<const uint4*>(row - W);
    const uint4 dn = *reinterpret_cast<const uint4*>(row + W);
    const uint32_t pw = x > 0 ? *reinterpret_cast<const uint32_t*>(row - 4) : 0u;
    const uint32_t nw = x + 16 < W ? *reinterpret_cast<const uint32_t*>(row + 16) : 0u;
    const uint32_t cw[6] = {pw, c.x, c.y, c.z, c.w, nw};
    const uint32_t uw[4] = {up.x, up.y, up.z, up.w}, dw[4] = {dn.x, dn.y, dn.z, dn.w};
    bool binary = known_binary;
    if (!binary) {
      uint32_t nb = nonbinary_bits(pw) | nonbinary_bits(nw);
#pragma unroll
      for (int j = 0; j < 4; ++j) nb |= nonbinary_bits(uw[j]) | nonbinary_bits(dw[j]) | nonbinary_bits(cw[j + 1]);
      binary = nb == 0;
    }
    uint32_t m[4];
    if (binary) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        m[j] = maj5(uw[j], dw[j], __funnelshift_l(cw[j], cw[j + 1], 8), __funnelshift_r(cw[j + 1], cw[j + 2], 8),
                    cw[j + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        m[j] = med5_bytes(uw[j], dw[j], __funnelshift_l(cw[j], cw[j + 1], 8), __funnelshift_r(cw[j + 1], cw[j + 2], 8),
                          cw[j + 1]);
    }
    uint4 out = make_uint4(m[0], m[1], m[2], m[3]);
    if (x == 0) out.x = (out.x & 0xffffff00u) | (c.x & 0xffu);                 // column 0 copied
    if (x + 16 == W) out.w = (out.w & 0x00ffffffu) | (c.w & 0xff000000u);      // column W-1 copied
    return out;
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
