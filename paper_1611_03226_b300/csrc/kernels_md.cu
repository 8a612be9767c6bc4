// Fused motion-detection actor: frame difference against the previous frame
// (delivered by a channel with one initial token, Sec. 4.1), threshold, 3x3
// erosion then dilation, and emission of one record per 16x16 tile with
// motion.  The record port has a variable rate (0..r_max records per firing,
// r_max = tiles per frame); a firing is enabled only while r_max record slots
// are free, so the number of firings is known only after the counts are.
//
// Kernels per step:
//   plan    (1 CTA)   candidate firings n_cand from the frame / count channels
//                     and the record space; zero the per-frame totals.
//   main    (persistent warps)  each warp walks the rows of one 32-row strip
//                     and 480-pixel column band for a chunk of consecutive
//                     frames, with the whole per-pixel pipeline in registers
//                     (see k_md_main).  When the previous-frame channel is the
//                     current-frame channel delayed by one token, the previous
//                     frame is read from the current channel's ring, where the
//                     same warp read it one frame earlier.
//   finish  (1 CTA)   exclusive scan of the per-frame record totals, the exact
//                     number of enabled firings, counter commit.
//   scatter (1 CTA per frame)  raster-order compaction of the tiles with
//                     count > 0 into the record ring, and the count token.
#include <algorithm>
#include "common.cuh"

namespace dfg {

constexpr int kMdThreads = 256;     // plan / finish / scatter kernels

// Motion bits of 4 pixels: bit i of the result is set iff |c_i - p_i| > thr,
// with the threshold test done bytewise: for d = |c - p| (per byte), d > thr
// iff d >= 128 or (d & 0x7f) + (127 - thr) carries into bit 7.  The four byte
// MSBs (bits 7, 15, 23, 31) are then gathered into bits 28..31 by one multiply.
__device__ __forceinline__ uint32_t motion_nibble_hi(uint32_t c, uint32_t p, uint32_t add4) {
  const uint32_t d = __vabsdiffu4(c, p);
  const uint32_t m = (d | ((d & 0x7f7f7f7fu) + add4)) & 0x80808080u;
  return m * 0x00204081u;                 // bits 28..31 = pixels 0..3
}

// 16 pixels (one tile column of a row) -> 16 motion bits, bit i = pixel i.
__device__ __forceinline__ uint32_t motion_bits16(uint4 c, uint4 p, uint32_t add4) {
  uint32_t acc = 0;
  acc = __funnelshift_l(motion_nibble_hi(c.w, p.w, add4), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.z, p.z, add4), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.y, p.y, add4), acc, 4);
  acc = __funnelshift_l(motion_nibble_hi(c.x, p.x, add4), acc, 4);
  return acc;
}

__global__ void k_md_plan(MdArgs a) {
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

size_t md_smem_bytes(int W) {
  (void)W;
  return 0;
}

constexpr int kMdRows = 32;               // strip height: two tile rows
constexpr int kMdWalk = kMdRows + 4;      // rows walked per strip (2-row halo each side)
constexpr int kMdPre = 4;                 // rows of loads in flight per lane
constexpr int kMdOwned = 30;              // tile columns owned per warp (lanes 1..30)
constexpr int kMdWarpsPerCta = 4;

// One warp = one worker.  Work unit = (32-row strip, band of 30 tile columns,
// chunk of consecutive frames).  Lane l covers tile column 30*band - 1 + l
// (lanes 0 and 31 are halo lanes that only supply neighbour bits).  For every
// frame of its chunk the warp walks the strip's rows plus a 2-row halo, each
// lane loading 16 bytes of the current and of the previous frame per row
// (coalesced 512-byte rows per warp), and keeps the bit-plane pipeline
//   b = |cur - prev| > thr  ->  erosion (3 rows)  ->  dilation (3 rows)  ->  popcount
// in registers; horizontal neighbours come from lane shuffles.  The previous
// frame of frame j is the current frame of j - 1 that the same warp just read,
// so it is served by L1/L2 and each frame byte is read from DRAM about once.
__global__ void __launch_bounds__(kMdWarpsPerCta * 32, 6) k_md_main(MdArgs a) {
  const MdPlanHdr pl = *a.plan;
  const uint64_t n = pl.n_cand;
  if (n == 0) return;
  const int W = a.W, H = a.H;
  const int lane = threadIdx.x & 31;
  const int cols = W / 16;                                    // tile columns
  const int bands = (cols + kMdOwned - 1) / kMdOwned;
  const int strips = (H + kMdRows - 1) / kMdRows;
  const uint32_t pairs = (uint32_t)(strips * bands);
  const uint32_t G = gridDim.x * kMdWarpsPerCta;              // workers
  uint32_t chunks = G / pairs;
  if (chunks < 1) chunks = 1;
  if (chunks > n) chunks = (uint32_t)n;
  const uint32_t units = pairs * chunks;
  const uint32_t add4 = 0x01010101u * (uint32_t)(127 - a.thr);
  for (uint32_t u = blockIdx.x * kMdWarpsPerCta + (threadIdx.x >> 5); u < units; u += G) {
    const uint32_t pair = u % pairs, chunk = u / pairs;
    const int strip = (int)(pair / bands), band = (int)(pair % bands);
    const uint64_t j0 = n * chunk / chunks, j1 = n * (chunk + 1) / chunks;
    const int col = band * kMdOwned - 1 + lane;               // this lane's tile column
    const bool col_in = col >= 0 && col < cols;
    const bool owned = lane >= 1 && lane <= kMdOwned && col_in;
    const int y0 = strip * kMdRows;
    const size_t col_off = (size_t)(col_in ? col : 0) * 16;
    for (uint64_t j = j0; j < j1; ++j) {
      const uint8_t* cur = slot_ptr(a.cur, pl.rd_cur0 + j) + col_off;
      const uint8_t* prv;
      if (a.dedup && j >= 1) prv = slot_ptr(a.cur, pl.rd_cur0 + j - 1) + col_off;
      else prv = slot_ptr(a.prev, pl.rd_prev0 + j) + col_off;
      uint4 cb[kMdPre], pb[kMdPre];
#pragma unroll
      for (int r = 0; r < kMdPre; ++r) {
        const int y = y0 - 2 + r;
        if (col_in && y >= 0 && y < H) {
          cb[r] = __ldg(reinterpret_cast<const uint4*>(cur + (size_t)y * W));
          pb[r] = __ldg(reinterpret_cast<const uint4*>(prv + (size_t)y * W));
        }
      }
      uint32_t hb1 = 0, hb2 = 0;        // horizontally eroded rows y-2, y-1
      uint32_t he1 = 0, he2 = 0;        // horizontally dilated erosion rows
      uint32_t cnt0 = 0, cnt1 = 0;      // tile counts of the two tile rows
#pragma unroll 1
      for (int rg = 0; rg < kMdWalk; rg += kMdPre) {
#pragma unroll
        for (int q = 0; q < kMdPre; ++q) {
          const int r = rg + q;
          const int y = y0 - 2 + r;
          const bool row_in = y >= 0 && y < H;
          uint32_t b = 0xffffu;                                  // outside: erosion border
          if (col_in && row_in) b = motion_bits16(cb[q], pb[q], add4);
          if (r + kMdPre < kMdWalk) {
            const int yn = y + kMdPre;
            if (col_in && yn >= 0 && yn < H) {
              cb[q] = __ldg(reinterpret_cast<const uint4*>(cur + (size_t)yn * W));
              pb[q] = __ldg(reinterpret_cast<const uint4*>(prv + (size_t)yn * W));
            }
          }
          // horizontal erosion: x holds pixels -1..16 of this lane in bits 0..17
          const uint32_t l = __shfl_up_sync(0xffffffffu, b, 1);
          const uint32_t rr = __shfl_down_sync(0xffffffffu, b, 1);
          const uint32_t x = ((rr & 1u) << 17) | (b << 1) | ((l >> 15) & 1u);
          const uint32_t hb = x & (x >> 1) & (x >> 2) & 0xffffu;
          // erosion of row y-1 (rows y-2, y-1, y); 0 outside the frame (dilation border)
          const int ye = y - 1;
          uint32_t e = 0;
          if (r >= 2 && col_in && ye >= 0 && ye < H) e = hb2 & hb1 & hb;
          hb2 = hb1;
          hb1 = hb;
          const uint32_t le = __shfl_up_sync(0xffffffffu, e, 1);
          const uint32_t re = __shfl_down_sync(0xffffffffu, e, 1);
          const uint32_t xe = ((re & 1u) << 17) | (e << 1) | ((le >> 15) & 1u);
          const uint32_t he = (xe | (xe >> 1) | (xe >> 2)) & 0xffffu;
          // dilation of row y-2 (erosion rows y-3, y-2, y-1), produced for r = 4 .. 35
          const int yo = y - 2;
          if (r >= 4 && yo < H) {
            const uint32_t pc = __popc(he2 | he1 | he);
            if (r - 4 < 16) cnt0 += pc;
            else cnt1 += pc;
          }
          he2 = he1;
          he1 = he;
        }
      }
      // rows y0 .. y0+31 were produced at r = 4 .. 35
      uint32_t nz = 0;
      const int ty0 = 2 * strip;
      if (owned) a.counts[j * a.n_tiles + (size_t)ty0 * a.tiles_x + col] = (uint16_t)cnt0;
      nz += __popc(__ballot_sync(0xffffffffu, owned && cnt0 > 0));
      if (ty0 + 1 < a.tiles_y) {
        if (owned) a.counts[j * a.n_tiles + (size_t)(ty0 + 1) * a.tiles_x + col] = (uint16_t)cnt1;
        nz += __popc(__ballot_sync(0xffffffffu, owned && cnt1 > 0));
      }
      if (lane == 0 && nz) atomicAdd(&a.frame_tot[j], nz);
    }
  }
}

__global__ void k_md_finish(MdArgs a) {
  uint64_t* frame_off = a.frame_off;
  __shared__ uint64_t sw[32];
  __shared__ uint64_t s_n;
  MdPlanHdr* pl = a.plan;
  const uint64_t n_cand = pl->n_cand;
  const uint64_t free_rec = pl->free_rec;
  if (threadIdx.x == 0) s_n = n_cand;
  __syncthreads();
  uint64_t carry = 0;
  for (uint64_t base = 0; base < n_cand; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t v = i < n_cand ? a.frame_tot[i] : 0;
    // exclusive scan (block)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t s = lane < nw ? sw[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) sw[lane] = s;
    }
    __syncthreads();
    const uint64_t off = carry + (wid ? sw[wid - 1] : 0) + x - v;
    const uint64_t tot = sw[nw - 1];
    __syncthreads();
    if (i < n_cand) {
      frame_off[i] = off;
      // firing i is enabled iff r_max record slots are free before it
      if (off + (uint64_t)a.n_tiles > free_rec) atomicMin((unsigned long long*)&s_n, i);
    }
    carry += tot;
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t n = s_n;
    const uint64_t used = n < n_cand ? frame_off[n] : carry;
    frame_off[n] = used;
    pl->n_cand = n;                 // the scatter kernel handles exactly n firings
    uint64_t* ctr = a.ctr;
    *rd_ptr(ctr, a.cur.id) = pl->rd_cur0 + n;
    *rd_ptr(ctr, a.prev.id) = pl->rd_prev0 + n;
    *wr_ptr(ctr, a.cnt.id) = pl->wr_cnt0 + n;
    *wr_ptr(ctr, a.rec.id) = pl->wr_rec0 + used;
    atomicAdd(&a.eng->fired_step, (unsigned long long)n);
    atomicAdd(&a.eng->fired_total, (unsigned long long)n);
  }
}

__global__ void __launch_bounds__(kMdThreads) k_md_scatter(MdArgs a) {
  const uint64_t* frame_off = a.frame_off;
  __shared__ uint32_t sw[32];
  const uint64_t j = blockIdx.x;
  const MdPlanHdr pl = *a.plan;
  if (j >= pl.n_cand) return;
  const int nt = a.n_tiles;
  const int per = (nt + kMdThreads - 1) / kMdThreads;
  const int t0 = threadIdx.x * per, t1 = min(nt, t0 + per);
  const uint16_t* cnt = a.counts + j * nt;
  uint32_t mine = 0;
  for (int t = t0; t < t1; ++t) mine += cnt[t] > 0;
  // exclusive scan of `mine` over the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? sw[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sw[lane] = s;
  }
  __syncthreads();
  uint64_t pos = pl.wr_rec0 + frame_off[j] + (wid ? sw[wid - 1] : 0) + x - mine;
  for (int t = t0; t < t1; ++t) {
    const uint32_t c = cnt[t];
    if (c > 0) {
      const uint32_t tx = t % a.tiles_x, ty = t / a.tiles_x;
      uint2 rec;
      rec.x = (16u * tx) | ((16u * ty) << 16);
      rec.y = c;
      *reinterpret_cast<uint2*>(slot_ptr(a.rec, pos)) = rec;
      ++pos;
    }
  }
  if (threadIdx.x == 0)
    *reinterpret_cast<uint32_t*>(slot_ptr(a.cnt, pl.wr_cnt0 + j)) = a.frame_tot[j];
}

static int g_md_blocks_per_sm = 0;

cudaError_t md_prepare(int W) {
  (void)W;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md_main,
                                                                kMdWarpsPerCta * 32, 0);
  if (e != cudaSuccess) return e;
  g_md_blocks_per_sm = per_sm > 0 ? per_sm : 1;
  return cudaSuccess;
}

cudaError_t launch_md_step(const MdArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0,
                           cudaEvent_t ev1) {
  k_md_plan<<<1, 256, 0, s>>>(a);
  if (ev0) cudaEventRecord(ev0, s);
  k_md_main<<<n_sm * (g_md_blocks_per_sm ? g_md_blocks_per_sm : 8), kMdWarpsPerCta * 32, 0, s>>>(a);
  if (ev1) cudaEventRecord(ev1, s);
  k_md_finish<<<1, 256, 0, s>>>(a);
  k_md_scatter<<<a.n_max, kMdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dfg
