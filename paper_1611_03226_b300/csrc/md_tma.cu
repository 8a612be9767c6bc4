// Main phase of the fused motion-detection actor (Sec. 4.1) with the frame
// rows staged in shared memory by the tensor memory accelerator (TMA).
//
// Used when the previous-frame channel carries the current-frame stream
// delayed by one token, so that every frame is read once per work unit.  A
// CTA takes one work unit at a time -- a 48-row strip of a panel of up to 4
// column bands (480 pixels each) over kTFrames consecutive frames j0 .. -- and
// walks the strip's rows plus a 2-row halo above and below in groups of
// kTRows rows:
//
//   producer warp   copies each row group of the frames the unit reads
//                   (j0-1 ..) into a ring of kTStages shared-memory stages.
//                   A box row is the panel's pixels plus one 16-pixel halo
//                   tile column on each side (1952 bytes for 4 bands), so the
//                   rows of a frame arrive as long contiguous runs; pixels
//                   outside the image arrive as zeros and are never used.
//   consumer warp (band b, pair q) runs the per-pixel pipeline for band b of
//                   the frame pair j0+2q, j0+2q+1 (previous frames j0+2q-1 and
//                   j0+2q) in registers: lane l holds the 16 pixels of tile
//                   column 30*(panel band) - 1 + l of both frames,
//                   bit-interleaved in one word (frame j0+2q+1 in the even
//                   bits, j0+2q in the odd bits), so that one funnel shift
//                   gives the horizontal neighbours of both frames.
//
// Each stage has a "full" barrier (the producer's expected byte count, which
// the TMA completes) and an "empty" barrier (one arrival per consumer warp).
// Every wait is bounded by the engine's wait limit; a wait that runs out
// records DF_ETIMEOUT, and the producer waits (again bounded) for its copies
// in flight before it leaves, so no copy lands in the shared memory of a CTA
// that has exited.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "md_dev.cuh"

namespace dfg {
namespace {

constexpr int kTRows = 4;                          // rows per stage
constexpr int kTStages = 3;
constexpr int kTFrames = 8;                        // frames per work unit
constexpr int kTSlots = kTFrames + 1;              // plus the previous frame of the first
constexpr int kTPanel = 4;                         // column bands per panel
constexpr int kTBand = kMdOwned * 16;              // pixels per band (480)
constexpr int kTGroups = kMdWalk / kTRows;
constexpr int kTPairs = kTFrames / 2;
constexpr int kTConsumers = kTPanel * kTPairs;
constexpr int kTThreads = (kTConsumers + 1) * 32;
constexpr int kTBarBytes = 128;                    // barriers, ahead of the stages
static_assert(kMdWalk % kTRows == 0 && 4 % kTRows == 0,
              "row groups tile the walk and the first 4 walk rows");
static_assert(2 * kTStages * sizeof(uint64_t) <= kTBarBytes, "barrier area");
static_assert(4 % kTRows == 0 && kMdWalk % kTRows == 0, "row groups tile the walk and its first 4 rows");

// Bytes of one frame's rows in a stage: kTRows rows of `pitch` bytes, padded
// to the 128-byte alignment a TMA destination needs.
__host__ __device__ constexpr int tma_slot_bytes(int pitch) { return (kTRows * pitch + 127) & ~127; }

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_done(uint32_t bar, uint32_t parity) {
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
// Wait until the barrier phase of the given parity has completed, at most
// limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit_ns) {
  if (mbar_done(bar, parity)) return true;
  const long long t0 = globaltimer_ns();
  while (!mbar_done(bar, parity))
    if (globaltimer_ns() - t0 > limit_ns) return false;
  return true;
}
// One 3-D tiled TMA load (x = pixel, y = row, z = ring slot) into shared memory.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Byte MSBs (bits 7, 15, 23, 31) set where |c - p| > t, all other bits clear
// (the bytewise test of ThrCode; HI selects the form for t >= 128).
template <bool HI>
__device__ __forceinline__ uint32_t over_msb(uint32_t c, uint32_t p, uint32_t add4) {
  const uint32_t d = __vabsdiffu4(c, p);
  const uint32_t s = (d & 0x7f7f7f7fu) + add4;
  return (HI ? (d & s) : (d | s)) & 0x80808080u;
}

// Motion bits of 4 pixels of frames A (previous word pa) and B (previous word
// a), interleaved in one byte: bit 2j = B pixel j, bit 2j + 1 = A pixel j.
// Two 32 x 32 -> 64-bit multiplies move A's byte MSBs by 26, 20, 14, 8 bits to
// 33, 35, 37, 39 and B's by 25, 19, 13, 7 bits to 32, 34, 36, 38; every
// partial product of A lands on an odd bit and of B on an even bit, all
// distinct, so the sum has no carries and bits 32..39 are the wanted byte.
constexpr uint32_t kGatherA = (1u << 26) | (1u << 20) | (1u << 14) | (1u << 8);
constexpr uint32_t kGatherB = (1u << 25) | (1u << 19) | (1u << 13) | (1u << 7);
template <bool HI>
__device__ __forceinline__ uint32_t pair_byte(uint32_t a, uint32_t pa, uint32_t b, uint32_t add4) {
  const uint64_t p = (uint64_t)over_msb<HI>(a, pa, add4) * kGatherA +
                     (uint64_t)over_msb<HI>(b, a, add4) * kGatherB;
  return (uint32_t)(p >> 32);                   // byte 0 is the result
}

// 16 pixels of frames A and B -> 32 bits, pixel i of B at bit 2i and of A at
// bit 2i + 1 (the byte of 16-byte word w goes to bits 8w .. 8w + 7).
template <bool HI>
__device__ __forceinline__ uint32_t pair_bits32(uint4 a, uint4 pa, uint4 b, uint32_t add4) {
  const uint32_t lo = __byte_perm(pair_byte<HI>(a.x, pa.x, b.x, add4),
                                  pair_byte<HI>(a.y, pa.y, b.y, add4), 0x0040);
  const uint32_t hi = __byte_perm(pair_byte<HI>(a.z, pa.z, b.z, add4),
                                  pair_byte<HI>(a.w, pa.w, b.w, add4), 0x0040);
  return __byte_perm(lo, hi, 0x5410);
}

// Per-lane state of one frame pair along the walk: the last two rows of the
// horizontal erosion (hb1 = previous row) and of the erosion output (he1), and
// the tile counts of the pair (3 tile rows in 10-bit fields; cn_all counts both
// frames, cn_lo frame B).
struct PairState {
  uint32_t hb1, hb2, he1, he2, cn_all, cn_lo;
};

// The 16-byte words of kTRows consecutive walked rows a lane reads from a
// stage: per row, frame A's previous frame, frame A and frame B.
struct StageRows {
  uint4 v[kTRows][3];
};
__device__ __forceinline__ void load_rows(const uint8_t* st, int step, int slot, StageRows& r) {
#pragma unroll
  for (int rr = 0; rr < kTRows; ++rr) {
    const uint8_t* row = st + rr * step;             // rows in walk order
    r.v[rr][0] = *reinterpret_cast<const uint4*>(row);
    r.v[rr][1] = *reinterpret_cast<const uint4*>(row + slot);
    r.v[rr][2] = *reinterpret_cast<const uint4*>(row + 2 * slot);
  }
}

// kTRows consecutive walked rows of one frame pair, from registers.
//   ROWS   the unit reaches outside the image vertically: per-row range tests
//   COLS   some lane's tile column is outside the image: lane masks
//   W0     walk row of the group's first row when it is below 4, else 4: the
//          erosion output starts at walk row 2 and the dilation output (tile
//          counts) at walk row 4
// Outside the image every pixel counts as motion for the erosion and as no
// motion for the dilation.
template <bool HI, bool ROWS, bool COLS, int W0>
__device__ __forceinline__ void pair_rows(const StageRows& r, int y_start, int dir, int H, bool col_in,
                                          uint32_t add4, uint32_t mul, PairState& p) {
#pragma unroll
  for (int rr = 0; rr < kTRows; ++rr) {
    const uint4 pv = r.v[rr][0], av = r.v[rr][1], bv = r.v[rr][2];
    const int y = y_start + dir * rr;
    uint32_t b = pair_bits32<HI>(av, pv, bv, add4);
    if (COLS && !col_in) b = 0xffffffffu;
    if (ROWS && (y < 0 || y >= H)) b = 0xffffffffu;
    const uint32_t bl = __shfl_up_sync(0xffffffffu, b, 1);
    const uint32_t br = __shfl_down_sync(0xffffffffu, b, 1);
    const uint32_t hrow = b & __funnelshift_l(bl, b, 2) & __funnelshift_r(b, br, 2);
    uint32_t e = 0;                                   // erosion, image row y - dir
    if (W0 + rr >= 2) {
      e = p.hb2 & p.hb1 & hrow;
      if (COLS && !col_in) e = 0;
      if (ROWS && (y - dir < 0 || y - dir >= H)) e = 0;
    }
    p.hb2 = p.hb1;
    p.hb1 = hrow;
    const uint32_t el = __shfl_up_sync(0xffffffffu, e, 1);
    const uint32_t er = __shfl_down_sync(0xffffffffu, e, 1);
    const uint32_t drow = e | __funnelshift_l(el, e, 2) | __funnelshift_r(e, er, 2);
    if (W0 + rr >= 4 && (!ROWS || y - 2 * dir < H)) {   // dilation, image row y - 2 dir
      const uint32_t o = p.he2 | p.he1 | drow;
      p.cn_all += (uint32_t)__popc(o) * mul;
      p.cn_lo += (uint32_t)__popc(o & 0x55555555u) * mul;
    }
    p.he2 = p.he1;
    p.he1 = drow;
  }
}

template <bool HI, int W0>
__device__ __forceinline__ void pair_rows_any(bool rows, bool cols, const StageRows& r, int y_start,
                                              int dir, int H, bool col_in, uint32_t add4, uint32_t mul,
                                              PairState& p) {
  if (rows) {
    if (cols) pair_rows<HI, true, true, W0>(r, y_start, dir, H, col_in, add4, mul, p);
    else pair_rows<HI, true, false, W0>(r, y_start, dir, H, col_in, add4, mul, p);
  } else {
    if (cols) pair_rows<HI, false, true, W0>(r, y_start, dir, H, col_in, add4, mul, p);
    else pair_rows<HI, false, false, W0>(r, y_start, dir, H, col_in, add4, mul, p);
  }
}

struct TmaUnit {
  int strip, panel;
  uint64_t j0;
  int nf;
};

__device__ __forceinline__ TmaUnit tma_unit(uint64_t u, uint32_t panels, uint32_t pairs, uint64_t n) {
  TmaUnit t;
  const uint32_t pair = (uint32_t)(u % pairs);
  t.strip = (int)(pair / panels);
  t.panel = (int)(pair % panels);
  t.j0 = (u / pairs) * kTFrames;
  const uint64_t left = n - t.j0;
  t.nf = left < (uint64_t)kTFrames ? (int)left : kTFrames;
  return t;
}

// Tile counts of one frame of the unit: 3 tile rows in 10-bit fields.
__device__ __forceinline__ void store_counts(const MdArgs& a, uint64_t j, uint32_t cn, int strip,
                                             int col, bool owned) {
  uint16_t* cnt = a.counts + j * a.n_tiles;
  const int ty0 = kMdTileRows * strip;
  uint32_t nz = 0;
#pragma unroll
  for (int tr = 0; tr < kMdTileRows; ++tr) {
    const uint32_t c = (cn >> (10 * tr)) & 0x3ffu;
    const bool in = owned && ty0 + tr < a.tiles_y;
    if (in) cnt[(size_t)(ty0 + tr) * a.tiles_x + col] = (uint16_t)c;
    nz += __popc(__ballot_sync(0xffffffffu, in && c));
  }
  if ((threadIdx.x & 31) == 0 && nz) atomicAdd(&a.frame_tot[j], nz);
}

template <bool HI>
__global__ void __launch_bounds__(kTThreads)
    k_md_main_tma(MdArgs a, MdTmaGeom geo, const __grid_constant__ CUtensorMap tm_unit,
                  const __grid_constant__ CUtensorMap tm_cur,
                  const __grid_constant__ CUtensorMap tm_prev) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int pitch = geo.pitch;                         // bytes per staged row
  const int slot_bytes = tma_slot_bytes(pitch);        // one frame's rows in a stage
  const int stage_bytes = kTSlots * slot_bytes;
  uint8_t* stages = smem + kTBarBytes;
  const uint32_t full0 = smem_addr(smem), empty0 = full0 + 8 * kTStages;
  __shared__ MdPlanHdr s_pl;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, kTConsumers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  griddep_wait();
  // one load of the plan per CTA (every CTA reads the same line)
  if (threadIdx.x == 0) s_pl = *a.plan;
  __syncthreads();
  const MdPlanHdr pl = s_pl;
  const uint64_t n = pl.n_cand;
  if (n == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cols = a.W / 16;
  const uint32_t bands = (uint32_t)((cols + kMdOwned - 1) / kMdOwned);
  const uint32_t panels = (bands + kTPanel - 1) / kTPanel;
  const uint32_t strips = (uint32_t)((a.H + kMdRows - 1) / kMdRows);
  const uint32_t pairs = strips * panels;
  const uint64_t units = (uint64_t)pairs * ((n + kTFrames - 1) / kTFrames);
  const long long limit = a.wait_limit_ns;

  if (warp == kTConsumers) {
    // ------------------------------------------------------- producer ----
    const uint64_t slot_cur0 = pl.rd_cur0 % a.cur.cap;
    const uint64_t slot_prev0 = pl.rd_prev0 % a.prev.cap;
    uint32_t g = 0;
    bool ok = true;
    for (uint64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const TmaUnit t = tma_unit(u, panels, pairs, n);
      // Frames j0-1 .. j0+nf-1 sit in slots z0 .. z0+nf of the current ring.
      // A full unit whose slots do not wrap at the ring's end comes in one copy;
      // otherwise (a short last unit, a wrap, or j0 = 0, where frame -1 is the
      // previous channel's initial token) one copy per frame.
      const uint64_t z0 = (t.j0 == 0) ? 0 : (slot_cur0 + t.j0 - 1) % a.cur.cap;
      const bool whole = t.j0 >= 1 && t.nf == kTFrames && z0 + (uint64_t)t.nf + 1 <= a.cur.cap &&
                         slot_bytes == kTRows * pitch;   // one box fills the slots without gaps
      const int copies = whole ? 1 : t.nf + 1;
      // bytes the copies deliver: kTRows rows of `pitch` per frame (the slot
      // padding is not written)
      const uint32_t bytes = (uint32_t)(whole ? kTSlots : t.nf + 1) * (uint32_t)(kTRows * pitch);
      const CUtensorMap* map = &tm_unit;
      int z = (int)z0;
      if (!whole) {                                  // this lane's frame j0 - 1 + lane
        map = &tm_cur;
        if (lane == 0 && t.j0 == 0) {
          map = &tm_prev;
          z = (int)slot_prev0;
        } else {
          uint64_t sl = slot_cur0 + t.j0 - 1 + lane;
          if (sl >= a.cur.cap) sl -= a.cur.cap;
          z = (int)sl;
        }
      }
      const int x = (t.panel * kTPanel * kTBand - 16) / 8;  // 64-bit elements; -2 for panel 0
      // Odd strips walk upwards, so that the rows two neighbouring strips share
      // are read by both at the same time (at the ends or at the starts of
      // their walks) while they run side by side.
      const bool up = t.strip & 1;
      const int y0 = up ? t.strip * kMdRows + kMdWalk - 2 - kTRows : t.strip * kMdRows - 2;
      const int dy = up ? -kTRows : kTRows;
      for (int grp = 0; grp < kTGroups; ++grp, ++g) {
        const uint32_t s = g % kTStages;
        if (g >= (uint32_t)kTStages && !mbar_wait(empty0 + 8 * s, ((g / kTStages) - 1) & 1, limit)) {
          if (lane == 0) set_status(a.eng, DF_ETIMEOUT, kWhereMdPipe);
          ok = false;
          break;
        }
        if (lane == 0) mbar_arrive_expect_tx(full0 + 8 * s, bytes);
        __syncwarp();
        if (lane < copies)
          tma_load_3d(smem_addr(stages + s * stage_bytes + lane * slot_bytes), map, x,
                      y0 + grp * dy, z, full0 + 8 * s);
      }
    }
    if (!ok) {
      // wait (bounded) for the copies still in flight before leaving
      const uint32_t first = g > (uint32_t)kTStages ? g - kTStages : 0;
      for (uint32_t i = first; i < g; ++i) mbar_wait(full0 + 8 * (i % kTStages), (i / kTStages) & 1, limit);
    }
    return;
  }

  // ----------------------------------------------------------- consumers ----
  const int pb = warp % kTPanel, q = warp / kTPanel;   // band in the panel, frame pair
  const uint32_t add4 = thr_code(a.thr).add4;
  const uint32_t lane_off = (uint32_t)(pb * kTBand + lane * 16);
  uint32_t g = 0;
  for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const TmaUnit t = tma_unit(u, panels, pairs, n);
    const int band = t.panel * kTPanel + pb;
    const int col = band * kMdOwned - 1 + lane;       // this lane's tile column
    const bool col_in = col >= 0 && col < cols;
    const bool owned = lane >= 1 && lane <= kMdOwned && col_in;
    const bool active = 2 * q < t.nf && band < (int)bands;
    const int ys = t.strip * kMdRows;
    // walked rows ys-2 .. ys+49 all inside the image / all lanes' columns inside
    const bool edge_rows = !(ys >= 2 && ys + kMdWalk - 2 <= a.H);
    const bool edge_cols = !(band >= 1 && (band + 1) * kMdOwned + 1 <= cols);
    const bool up = t.strip & 1;                       // walk direction (see the producer)
    const int dir = up ? -1 : 1;
    PairState p{0, 0, 0, 0, 0, 0};
    for (int grp = 0; grp < kTGroups; ++grp, ++g) {
      const uint32_t s = g % kTStages;
      if (!mbar_wait(full0 + 8 * s, (g / kTStages) & 1, limit)) {
        if (lane == 0) set_status(a.eng, DF_ETIMEOUT, kWhereMdPipe);
        return;
      }
      // The lane's words of the stage go to registers first and the stage is
      // handed back to the producer before the per-pixel work, so that the
      // copies of the next groups are in flight while it runs.
      StageRows r;
      if (active) {
        // the first row of this group in walk order, and the step between rows
        const uint8_t* st = stages + s * stage_bytes + (2 * q) * slot_bytes + lane_off +
                            (up ? (kTRows - 1) * pitch : 0);
        load_rows(st, up ? -pitch : pitch, slot_bytes, r);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * s);
      if (active) {
        const int y_start = up ? ys + kMdWalk - 3 - grp * kTRows : ys - 2 + grp * kTRows;
        // 10-bit count field of the tile row these dilation rows fall in
        const int tr = max(grp * kTRows - 4, 0) >> 4;
        uint32_t mul;                                  // 1 << (10 * field)
        asm("mov.b32 %0, %1;" : "=r"(mul) : "r"(1u << (10 * (up ? kMdTileRows - 1 - tr : tr))));
        const int w0 = grp * kTRows;                   // walk row of the group's first row
        if (w0 >= 4)
          pair_rows_any<HI, 4>(edge_rows, edge_cols, r, y_start, dir, a.H, col_in, add4, mul, p);
        else if (w0 == 0)
          pair_rows_any<HI, 0>(edge_rows, edge_cols, r, y_start, dir, a.H, col_in, add4, mul, p);
        else if (w0 == 2 && kTRows <= 2)
          pair_rows_any<HI, 2>(edge_rows, edge_cols, r, y_start, dir, a.H, col_in, add4, mul, p);
        else if (w0 == 1 && kTRows == 1)
          pair_rows_any<HI, 1>(edge_rows, edge_cols, r, y_start, dir, a.H, col_in, add4, mul, p);
        else if (kTRows == 1)
          pair_rows_any<HI, 3>(edge_rows, edge_cols, r, y_start, dir, a.H, col_in, add4, mul, p);
      }
    }
    if (active) {
      store_counts(a, t.j0 + 2 * q, p.cn_all - p.cn_lo, t.strip, col, owned);
      if (2 * q + 1 < t.nf) store_counts(a, t.j0 + 2 * q + 1, p.cn_lo, t.strip, col, owned);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Frames of a ring as a 3-D tensor of 64-bit elements (8 pixels): x = W / 8
// per row, y = row, z = slot; a box is `px` pixels of kTRows rows and `frames`
// consecutive slots.
bool encode_frames(CUtensorMap* m, const ChanDesc& c, int W, int H, int px, int frames) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((uint64_t)W * H != c.tok || c.cap > 0x7fffffffull || W % 8 || px % 8 || px / 8 > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W / 8, (cuuint64_t)H, (cuuint64_t)c.cap};
  const cuuint64_t strides[2] = {(cuuint64_t)W, (cuuint64_t)W * H};
  const cuuint32_t box[3] = {(cuuint32_t)px / 8, kTRows, (cuuint32_t)frames};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, c.ring, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void (*const g_kern[2])(MdArgs, MdTmaGeom, const CUtensorMap, const CUtensorMap, const CUtensorMap) = {
    k_md_main_tma<false>, k_md_main_tma<true>};

}  // namespace

cudaError_t md_tma_prepare(const MdArgs& a, MdTma* t) {
  t->ok = 0;
  if (!a.dedup || (uintptr_t)a.cur.ring % 16 || (uintptr_t)a.prev.ring % 16) return cudaSuccess;
  const int cols = a.W / 16;
  const int bands = (cols + kMdOwned - 1) / kMdOwned;
  const int pb = std::min(bands, kTPanel);               // bands per panel
  const int px = pb * kTBand + 32;                       // staged pixels per row
  t->geo.pitch = px;
  t->smem = (size_t)kTBarBytes + (size_t)kTStages * kTSlots * tma_slot_bytes(px);
  if (!encode_frames(&t->unit, a.cur, a.W, a.H, px, kTSlots) ||
      !encode_frames(&t->cur, a.cur, a.W, a.H, px, 1) || !encode_frames(&t->prev, a.prev, a.W, a.H, px, 1))
    return cudaSuccess;                                  // the register-staged kernel serves
  auto k = g_kern[a.thr >= 128 ? 1 : 0];
  // allow the largest dynamic size this device gives a block next to the
  // kernel's static shared memory
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  if (t->smem + fa.sharedSizeBytes > (size_t)optin) return cudaSuccess;   // the register-staged kernel serves
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTThreads, t->smem);
  if (e != cudaSuccess) return e;
  t->blocks_per_sm = per_sm > 0 ? per_sm : 1;
  t->ok = 1;
  return cudaSuccess;
}

cudaError_t launch_md_main_tma(const MdArgs& a, const MdTma& t, int n_sm, cudaStream_t s, bool pdl) {
  return launch_k(pdl, g_kern[a.thr >= 128 ? 1 : 0], dim3(n_sm * t.blocks_per_sm), dim3(kTThreads), t.smem,
                  s, a, t.geo, t.unit, t.cur, t.prev);
}

}  // namespace dfg
