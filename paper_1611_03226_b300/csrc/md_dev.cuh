// Device-side phases of the fused motion-detection actor: frame difference against the previous frame
// (delivered by a channel with one initial token, Sec. 4.1), threshold, 3x3
// erosion then dilation, and emission of one record per 16x16 tile with
// motion.  The record port has a variable rate (0..r_max records per firing,
// r_max = tiles per frame); a firing is enabled only while r_max record slots
// are free, so the number of firings is known only after the counts are.
//
// Kernels per step:
//   plan    (1 CTA)   candidate firings n_cand from the frame / count channels
//                     and the record space; zero the per-frame totals.
//   main    (persistent warps)  each warp walks the rows of one 48-row strip
//                     and 480-pixel column band for a chunk of 8 consecutive
//                     frames, with the whole per-pixel pipeline in registers
//                     (see md_unit).  When the previous-frame channel is the
//                     current-frame channel delayed by one token, each frame
//                     row is loaded once and serves both frames that use it.
//   emit    (1 CTA per frame)  exclusive scan of the per-frame record totals,
//                     the exact number of enabled firings, raster-order
//                     compaction of the tiles with count > 0 into the record
//                     ring, the count token; block 0 commits the counters.
#pragma once
#include <algorithm>
#include "common.cuh"

namespace dfg {


constexpr int kMdThreads = 256;     // plan and emit kernels

// Bytewise threshold test.  For d = |c - p| (per byte) and threshold t:
//   t <= 127:  d > t  iff  d >= 128  or  (d & 0x7f) + (127 - t) carries into bit 7;
//   t >= 128:  d > t  iff  d >= 128  and (d & 0x7f) + (255 - t) carries into bit 7.
// add4 holds (127 - t) mod 128 in every byte; or4 is 0x80808080 when either
// condition suffices (t <= 127) and 0 when both are needed (t >= 128).
struct ThrCode {
  uint32_t add4, or4;
};
__host__ __device__ inline ThrCode thr_code(int t) {
  return {0x01010101u * (uint32_t)((127 - t) & 127), t <= 127 ? 0x80808080u : 0u};
}
// Byte MSBs (bits 7, 15, 23, 31) set where d > t, all other bits clear.
__device__ __forceinline__ uint32_t over_thr_msb(uint32_t d, ThrCode k) {
  const uint32_t s = (d & 0x7f7f7f7fu) + k.add4;
  return ((d & s) | ((d | s) & k.or4)) & 0x80808080u;
}

// Motion bits of 4 pixels: the four byte MSBs of the threshold test are
// gathered into bits 28..31 (pixels 0..3) by one multiply.
__device__ __forceinline__ uint32_t motion_nibble_hi(uint32_t c, uint32_t p, ThrCode k) {
  return over_thr_msb(__vabsdiffu4(c, p), k) * 0x00204081u;
}

__device__ inline void md_plan_dev(const MdArgs& a) {
  __shared__ uint64_t s_n;
  if (threadIdx.x == 0) {
    uint64_t* ctr = a.ctr;
    const uint64_t rdc = *rd_ptr(ctr, a.cur.id), wrc = *wr_ptr(ctr, a.cur.id);
    const uint64_t rdp = *rd_ptr(ctr, a.prev.id), wrp = *wr_ptr(ctr, a.prev.id);
    const uint64_t wrr = *wr_ptr(ctr, a.rec.id), rdr = *rd_ptr(ctr, a.rec.id);
    const uint64_t wrn = *wr_ptr(ctr, a.cnt.id), rdn = *rd_ptr(ctr, a.cnt.id);
    uint64_t n = wrc - rdc;
    n = min(n, wrp - rdp);
    n = min(n, a.cnt.cap - (wrn - rdn));
    n = min(n, (uint64_t)a.n_max);
    const uint64_t free_rec = a.rec.cap - (wrr - rdr);
    if (free_rec < (uint64_t)a.n_tiles) n = 0;
    MdPlanHdr* pl = a.plan;
    pl->n_cand = n;
    pl->rd_cur0 = rdc;
    pl->rd_prev0 = rdp;
    pl->wr_rec0 = wrr;
    pl->wr_cnt0 = wrn;
    pl->free_rec = free_rec;
    s_n = n;
  }
  __syncthreads();
  for (uint64_t j = threadIdx.x; j < s_n; j += blockDim.x) a.frame_tot[j] = 0;
}


constexpr int kMdTileRows = 3;           // tile rows per strip
constexpr int kMdRows = 16 * kMdTileRows; // strip height
constexpr int kMdWalk = kMdRows + 4;      // rows walked per strip (2-row halo each side)
constexpr int kMdOwned = 30;              // tile columns owned per warp (lanes 1..30)
constexpr int kMdWarpsPerCta = 4;
constexpr int kMdFrames = 8;              // frames per work unit

// 16 pixels (one tile column of one row) -> 16 motion bits, bit i = pixel i.
__device__ __forceinline__ uint32_t motion_bits16(uint4 c, uint4 p, ThrCode tc) {
  uint32_t acc = 0;
  acc = __funnelshift_l(motion_nibble_hi(c.w, p.w, tc), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.z, p.z, tc), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.y, p.y, tc), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.x, p.x, tc), acc, 4);
  return acc;
}

// 16-byte row load; NC selects the read-only (non-coherent) path, valid only
// when no CTA of the same launch writes the ring.
template <bool NC>
__device__ __forceinline__ uint4 ld16(const uint8_t* p) {
  if constexpr (NC) return __ldg(reinterpret_cast<const uint4*>(p));
  else return *reinterpret_cast<const uint4*>(p);
}

__device__ __forceinline__ const uint8_t* frame_at(const ChanDesc& c, uint64_t slot0, uint64_t j) {
  uint64_t s = slot0 + j;
  if (s >= c.cap) s -= c.cap;
  return c.ring + s * c.tok;
}

// Two frames' 16-pixel rows packed in one word (frame A in bits 0..15, frame B
// in bits 16..31).  Horizontal 3-neighbourhoods of both halves at once: pixel i
// combines pixels i-1, i, i+1, where pixel -1 is bit 15 (31) of the left lane's
// word and pixel 16 is bit 0 (16) of the right lane's word.
__device__ __forceinline__ uint32_t left_nb(uint32_t v, uint32_t left) {     // pixel i-1 at bit i
  return ((v << 1) & 0xfffefffeu) | ((left >> 15) & 0x00010001u);
}
__device__ __forceinline__ uint32_t right_nb(uint32_t v, uint32_t right) {   // pixel i+1 at bit i
  return ((v >> 1) & 0x7fff7fffu) | ((right << 15) & 0x80008000u);
}

// One warp = one worker.  Work unit = (48-row strip, band of 30 tile columns,
// chunk of up to F consecutive frames, F even).  Lane l covers tile column
// 30*band - 1 + l; lanes 0 and 31 are halo lanes that only supply neighbour
// bits.  The warp walks the strip's rows plus a 2-row halo; for every row it
// reads that row of frames j0-1 .. j0+F-1 once (one 16-byte load per lane and
// frame, 512 contiguous bytes per warp), and each loaded row serves as the
// current row of frame j and the previous row of frame j+1.  The pipeline
//   b = |cur - prev| > thr  ->  erosion (3 rows)  ->  dilation (3 rows)  ->  popcount
// runs in registers on pairs of frames packed into one word; horizontal
// neighbour bits come from lane shuffles.  With a previous-frame channel that
// is not the delayed current channel, F = 2 with a separate previous row per
// frame.
template <int F, bool NC>
__device__ inline void md_unit(const MdArgs& a, uint64_t slot_cur0, uint64_t slot_prev0, int strip,
                        int band, uint64_t j0, int nf, ThrCode tc) {
  static_assert(F % 2 == 0, "frames are processed in pairs");
  constexpr int NP = F / 2;
  const int W = a.W, H = a.H;
  const int lane = threadIdx.x & 31;
  const int cols = W / 16;
  const int col = band * kMdOwned - 1 + lane;                // this lane's tile column
  const bool col_in = col >= 0 && col < cols;
  const bool owned = lane >= 1 && lane <= kMdOwned && col_in;
  const int y0 = strip * kMdRows;
  const size_t col_off = (size_t)(col_in ? col : 0) * 16;
  // Row sources.  F > 2 (shared previous rows, ring < 2 GiB): frame t of the
  // unit is at cbase + coff[t]; the previous frame of frame 0 is at p0.  F == 2:
  // explicit pointers for both frames and both previous frames.
  const uint8_t* cbase = frame_at(a.cur, slot_cur0, j0);
  int32_t coff[F];
#pragma unroll
  for (int t = 0; t < F; ++t) {
    const uint8_t* f = frame_at(a.cur, slot_cur0, j0 + (t < nf ? t : 0));
    coff[t] = (int32_t)(f - cbase);
  }
  const uint8_t* p0 = (a.dedup && j0 >= 1) ? frame_at(a.cur, slot_cur0, j0 - 1)
                                           : frame_at(a.prev, slot_prev0, j0);
  const uint8_t* p1 = nullptr;               // previous frame of frame 1 when not shared
  if constexpr (F == 2) {
    p1 = a.dedup ? frame_at(a.cur, slot_cur0, j0) : frame_at(a.prev, slot_prev0, j0 + (nf > 1 ? 1 : 0));
  }
  uint32_t hb1[NP], hb2[NP], he1[NP], he2[NP], cn[F];
#pragma unroll
  for (int q = 0; q < NP; ++q) hb1[q] = hb2[q] = he1[q] = he2[q] = 0;
#pragma unroll
  for (int t = 0; t < F; ++t) cn[t] = 0;
  // rows are software-pipelined: row r+1's loads are issued before row r is processed
  uint4 qc[F], qp0, qp1, nc[F], np0, np1;
  auto load_row = [&](int rr, uint4 (&c)[F], uint4& p0v, uint4& p1v) {
    const int yy = y0 - 2 + rr;
    const bool l = col_in && yy >= 0 && yy < H && rr < kMdWalk;
    const size_t o = (size_t)yy * W + col_off;
    const uint8_t* crow = cbase + o;
#pragma unroll
    for (int t = 0; t < F; ++t) {
      c[t] = make_uint4(0, 0, 0, 0);
      if (l && t < nf) c[t] = ld16<NC>(crow + coff[t]);
    }
    p0v = p1v = make_uint4(0, 0, 0, 0);
    if (l) p0v = ld16<NC>(p0 + o);
    if constexpr (F == 2) {
      if (l && nf > 1) p1v = ld16<NC>(p1 + o);
    }
  };
  load_row(0, qc, qp0, qp1);
#pragma unroll 1
  for (int r = 0; r < kMdWalk; ++r) {
    const int y = y0 - 2 + r;
    const bool ld = col_in && y >= 0 && y < H;
    load_row(r + 1, nc, np0, np1);
    const int ye = y - 1, yo = y - 2;
    const bool e_in = r >= 2 && col_in && ye >= 0 && ye < H;
    const bool o_in = r >= 4 && yo < H;
    const int sh = 10 * ((r - 4) >> 4);              // 10-bit count field of this tile row
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int ta = 2 * q, tb = 2 * q + 1;
      const uint4 pa = ta == 0 ? qp0 : qc[ta - 1];
      const uint4 pb = F == 2 ? qp1 : qc[ta];
      const uint32_t b = ld ? (motion_bits16(qc[ta], pa, tc) | (motion_bits16(qc[tb], pb, tc) << 16))
                            : 0xffffffffu;
      const uint32_t bl = __shfl_up_sync(0xffffffffu, b, 1);
      const uint32_t br = __shfl_down_sync(0xffffffffu, b, 1);
      const uint32_t hrow = b & left_nb(b, bl) & right_nb(b, br);
      const uint32_t e = e_in ? (hb2[q] & hb1[q] & hrow) : 0u;
      hb2[q] = hb1[q];
      hb1[q] = hrow;
      const uint32_t el = __shfl_up_sync(0xffffffffu, e, 1);
      const uint32_t er = __shfl_down_sync(0xffffffffu, e, 1);
      const uint32_t drow = e | left_nb(e, el) | right_nb(e, er);
      if (o_in) {
        const uint32_t o = he2[q] | he1[q] | drow;
        cn[ta] += (uint32_t)__popc(o & 0xffffu) << sh;
        cn[tb] += (uint32_t)__popc(o >> 16) << sh;
      }
      he2[q] = he1[q];
      he1[q] = drow;
    }
#pragma unroll
    for (int t = 0; t < F; ++t) qc[t] = nc[t];
    qp0 = np0;
    qp1 = np1;
  }
  // kMdTileRows tile rows per lane and frame (counts <= 256 in 10-bit fields)
  const int ty0 = kMdTileRows * strip;
#pragma unroll
  for (int t = 0; t < F; ++t) {
    if (t >= nf) break;
    const uint64_t j = j0 + t;
    uint16_t* cnt = a.counts + j * a.n_tiles;
    uint32_t nz = 0;
#pragma unroll
    for (int tr = 0; tr < kMdTileRows; ++tr) {
      const uint32_t c = (cn[t] >> (10 * tr)) & 0x3ffu;
      const bool in = owned && ty0 + tr < a.tiles_y;
      if (in) cnt[(size_t)(ty0 + tr) * a.tiles_x + col] = (uint16_t)c;
      nz += __popc(__ballot_sync(0xffffffffu, in && c));
    }
    if (lane == 0 && nz) atomicAdd(&a.frame_tot[j], nz);
  }
}

template <int F, bool NC>
__device__ inline void md_main_dev(const MdArgs& a, Grid g) {
  const int wpc = blockDim.x >> 5;                           // warps per CTA
  __shared__ MdPlanHdr s_pl;
  __syncthreads();                    // s_pl may still be read by a previous phase
  if (threadIdx.x == 0) s_pl = *a.plan;
  __syncthreads();
  const MdPlanHdr pl = s_pl;
  const uint64_t n = pl.n_cand;
  if (n == 0) return;
  const int cols = a.W / 16;
  const int bands = (cols + kMdOwned - 1) / kMdOwned;
  const int strips = (a.H + kMdRows - 1) / kMdRows;
  const uint32_t pairs = (uint32_t)(strips * bands);
  const uint64_t chunks = (n + F - 1) / F;
  const uint64_t units = pairs * chunks;
  const uint64_t G = (uint64_t)g.n * wpc;
  const ThrCode tc = thr_code(a.thr);
  const uint64_t slot_cur0 = pl.rd_cur0 % a.cur.cap, slot_prev0 = pl.rd_prev0 % a.prev.cap;
  for (uint64_t u = g.b * (uint64_t)wpc + (threadIdx.x >> 5); u < units; u += G) {
    const uint32_t pair = (uint32_t)(u % pairs);
    const uint64_t chunk = u / pairs;
    const uint64_t j0 = chunk * F;
    const uint64_t left = n - j0;
    const int nf = left < (uint64_t)F ? (int)left : F;
    md_unit<F, NC>(a, slot_cur0, slot_prev0, (int)(pair / bands), (int)(pair % bands), j0, nf, tc);
  }
}

// Record emission for frame j (one CTA): the exclusive scan of the per-frame
// record totals gives the frame's record offset and the exact number of enabled
// firings n (firing i is enabled iff r_max record slots are free before it);
// frames j < n scatter their records in raster order and their count token.
// The CTA with lead = true commits the counters.
__device__ inline void md_emit_frame(const MdArgs& a, uint64_t j, bool lead) {
  __shared__ uint64_t sw[32];
  __shared__ uint32_t sw32[32];
  __shared__ unsigned long long s_n;
  __shared__ uint64_t s_off, s_used;
  __shared__ MdPlanHdr s_pl;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // The loads of this frame's tile counts and of the first frame totals are
  // issued first: neither depends on the plan (frames past the candidates are
  // masked later), so their latency overlaps the plan's.
  // Tiles: warp w takes a contiguous run, 8 per lane per step (one 16-byte
  // load); the first kCache steps stay in registers for both passes.
  const int nt = a.n_tiles;
  const uint16_t* cnt = a.counts + j * nt;
  const bool vec = (nt % 8) == 0;                          // 16-byte aligned groups of 8 counts
  const int per_lane = vec ? 8 : 1;
  const int step = 32 * per_lane;                          // tiles per warp and step
  const int run = ((nt + nw * step - 1) / (nw * step)) * step;
  const int r0 = wid * run, r1 = min(nt, r0 + run);
  constexpr int kCache = 4;
  auto load_q = [&](int t) {
    uint4 q = make_uint4(0, 0, 0, 0);
    if (t < r1) {
      if (vec) q = *reinterpret_cast<const uint4*>(cnt + t);
      else q.x = cnt[t];
    }
    return q;
  };
  uint4 qc[kCache];
#pragma unroll
  for (int i = 0; i < kCache; ++i) qc[i] = load_q(r0 + i * step + lane * per_lane);
  // Frame totals: thread t takes kFr consecutive frames per pass.
  constexpr int kFr = 4;
  const uint64_t chunk = (uint64_t)kFr * blockDim.x;
  uint32_t tv[kFr];
#pragma unroll
  for (int q = 0; q < kFr; ++q) {
    const uint64_t i = (uint64_t)threadIdx.x * kFr + q;
    tv[q] = i < a.n_max ? a.frame_tot[i] : 0u;
  }
  // one load of the plan per CTA (every CTA of the phase reads the same line)
  if (threadIdx.x == 0) {
    s_pl = *a.plan;
    s_n = s_pl.n_cand;
    s_off = 0;
  }
  __syncthreads();
  const MdPlanHdr pl = s_pl;
  const uint64_t n_cand = pl.n_cand;
  if (j > 0 && j >= n_cand) return;                        // no such candidate frame

  // Exclusive scan of the frame totals: frame i's first record, and the
  // enabled firings (firing i needs r_max free record slots before it).
  uint64_t carry = 0;
  for (uint64_t base = 0; base < n_cand; base += chunk) {
    if (base > 0) {
#pragma unroll
      for (int q = 0; q < kFr; ++q) {
        const uint64_t i = base + (uint64_t)threadIdx.x * kFr + q;
        tv[q] = i < a.n_max ? a.frame_tot[i] : 0u;
      }
    }
    const uint64_t i0 = base + (uint64_t)threadIdx.x * kFr;
    uint64_t mine = 0;
#pragma unroll
    for (int q = 0; q < kFr; ++q) mine += i0 + q < n_cand ? tv[q] : 0u;
    uint64_t x = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t t = lane < nw ? sw[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) sw[lane] = t;
    }
    __syncthreads();
    uint64_t off = carry + (wid ? sw[wid - 1] : 0) + x - mine;
    const uint64_t tot = sw[nw - 1];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kFr; ++q) {
      const uint64_t i = i0 + q;
      if (i < n_cand) {
        if (off + (uint64_t)a.n_tiles > pl.free_rec) atomicMin(&s_n, (unsigned long long)i);
        if (i == j) s_off = off;
        if (lead) a.frame_off[i] = off;
        off += tv[q];
      }
    }
    carry += tot;
  }
  __syncthreads();
  const uint64_t n = s_n;
  if (lead && threadIdx.x == 0) s_used = n < n_cand ? a.frame_off[n] : carry;   // records of frames < n
  __syncthreads();
  if (lead && threadIdx.x == 0) {
    uint64_t* ctr = a.ctr;
    *rd_ptr(ctr, a.cur.id) = pl.rd_cur0 + n;
    *rd_ptr(ctr, a.prev.id) = pl.rd_prev0 + n;
    *wr_ptr(ctr, a.cnt.id) = pl.wr_cnt0 + n;
    *wr_ptr(ctr, a.rec.id) = pl.wr_rec0 + s_used;
    atomicAdd(&a.eng->fired_total, (unsigned long long)n);
  }
  if (j >= n) return;

  // Raster-order compaction of the tiles of frame j with count > 0: pass 1
  // counts each warp's records, a block scan gives each warp its first record,
  // pass 2 writes the records (a lane's in order after those of the lanes
  // below it).
  auto counts8 = [&](const uint4 q, uint32_t (&c)[8]) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
  };
  // step i's counts: registers for the first kCache steps, else a new load
  // (the cached loop is unrolled so that qc is indexed by constants)
  auto for_steps = [&](auto&& f) {
    const int steps = r1 > r0 ? (r1 - r0 + step - 1) / step : 0;
#pragma unroll
    for (int i = 0; i < kCache; ++i)
      if (i < steps) f(i, qc[i]);
    for (int i = kCache; i < steps; ++i) f(i, load_q(r0 + i * step + lane * per_lane));
  };
  uint32_t mine = 0;
  for_steps([&](int, const uint4 q) {
    uint32_t c[8];
    counts8(q, c);
#pragma unroll
    for (int k = 0; k < 8; ++k) mine += c[k] != 0;
  });
  const uint32_t warp_tot = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) sw32[wid] = warp_tot;
  __syncthreads();
  if (wid == 0) {
    uint32_t t = lane < nw ? sw32[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) sw32[lane] = t;                         // inclusive
  }
  __syncthreads();
  // ring slot of the frame's first record (records of one frame fit the ring,
  // so one subtraction wraps every slot below)
  const uint64_t slot0 = (pl.wr_rec0 + s_off) % a.rec.cap;
  uint64_t next = (wid ? sw32[wid - 1] : 0);               // records before this step
  for_steps([&](int i, const uint4 q) {
    uint32_t c[8];
    counts8(q, c);
    const int t0 = r0 + i * step + lane * per_lane;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) m += c[k] != 0;
    uint32_t incl = m;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint64_t idx = next + incl - m;
    next += __shfl_sync(0xffffffffu, incl, 31);
    if (m) {
      uint32_t ty = (uint32_t)t0 / (uint32_t)a.tiles_x, tx = (uint32_t)t0 - ty * (uint32_t)a.tiles_x;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (c[k]) {
          uint64_t slot = slot0 + idx;
          if (slot >= a.rec.cap) slot -= a.rec.cap;
          uint2 rec;
          rec.x = (16u * tx) | ((16u * ty) << 16);
          rec.y = c[k];
          *reinterpret_cast<uint2*>(a.rec.ring + slot * a.rec.tok) = rec;
          ++idx;
        }
        if (++tx == (uint32_t)a.tiles_x) {
          tx = 0;
          ++ty;
        }
      }
    }
  });
  if (threadIdx.x == 0)
    *reinterpret_cast<uint32_t*>(slot_ptr(a.cnt, pl.wr_cnt0 + j)) = a.frame_tot[j];
}

// Emission phase over a virtual grid: one CTA per frame (block 0 commits).
__device__ inline void md_emit_dev(const MdArgs& a, Grid g) {
  const uint64_t n = a.plan->n_cand;
  const uint64_t span = n > 0 ? n : 1;
  for (uint64_t j = g.b; j < span; j += g.n) {
    md_emit_frame(a, j, j == 0);
    __syncthreads();
  }
}

}  // namespace dfg
