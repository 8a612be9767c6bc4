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
//   main    (1 CTA/SM, persistent)  work = (16-row strip, frame) pairs in
//                     strip-major order, split evenly over the CTAs.  Each
//                     strip of the current frame (plus a 2-row halo) is copied
//                     into shared memory by cp.async.bulk on an mbarrier
//                     pipeline of 4 stages.  When the previous-frame channel is
//                     the current-frame channel delayed by one token, the
//                     previous frame's strip is the stage just consumed, so each
//                     frame byte is read from HBM once.  Pixels are thresholded
//                     4 at a time into 32-bit bit planes; erosion and dilation
//                     are shifts, ANDs and ORs on the bit planes; popcounts give
//                     the tile counts.
//   finish  (1 CTA)   exclusive scan of the per-frame record totals, the exact
//                     number of enabled firings, counter commit.
//   scatter (1 CTA per frame)  raster-order compaction of the tiles with
//                     count > 0 into the record ring, and the count token.
#include <algorithm>
#include "common.cuh"

namespace dfg {

constexpr int kRH = 16;               // strip rows = one tile row
constexpr int kBufRows = kRH + 4;     // plus two halo rows above and below
constexpr int kStages = 4;
constexpr int kMdThreads = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false when `limit_ns` passed without the phase completing.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 pixels of current and previous frame -> 16 motion bits (bit i = pixel i).
__device__ __forceinline__ uint32_t motion_bits16(uint4 c, uint4 p, uint32_t thr4) {
  const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
  const uint32_t pw[4] = {p.x, p.y, p.z, p.w};
  uint32_t out = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t d = __vabsdiffu4(cw[i], pw[i]);
    const uint32_t m = __vcmpgtu4(d, thr4);           // 0xff in every byte with d > thr
    // gather the four byte MSBs (bits 7,15,23,31) into bits 28..31
    const uint32_t nib = ((m & 0x80808080u) * 0x00204081u) >> 28;
    out |= nib << (4 * i);
  }
  return out;
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
  const size_t words = W / 32;
  const size_t stage = ((size_t)kBufRows * W + 127) / 128 * 128;
  return kStages * stage + (2 * kBufRows + kRH) * words * 4 + kStages * 8 + 16;
}

__global__ void __launch_bounds__(kMdThreads, 1) k_md_main(MdArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int s_abort;
  const MdPlanHdr pl = *a.plan;
  const uint64_t n = pl.n_cand;
  if (n == 0) return;
  const int W = a.W, H = a.H, words = a.words;
  const size_t stage_bytes = ((size_t)kBufRows * W + 127) / 128 * 128;
  uint8_t* stages = smem;
  uint32_t* bw = reinterpret_cast<uint32_t*>(smem + kStages * stage_bytes);
  uint32_t* ew = bw + kBufRows * words;
  uint32_t* pc = ew + kBufRows * words;
  uint64_t* bars = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(pc + kRH * words) + 7) & ~uintptr_t(7));

  const uint64_t total = (uint64_t)a.strips * n;
  const uint64_t first = total * blockIdx.x / gridDim.x;
  const uint64_t last = total * (blockIdx.x + 1) / gridDim.x;
  if (first >= last) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();

  const uint32_t thr4 = 0x01010101u * (uint32_t)a.thr;
  const int chunks_row = W / 16;
  auto needs_prev_load = [&](uint64_t item) {
    return !a.dedup || item == first || (item % n) == 0;
  };
  // producer state (thread 0)
  uint64_t p_item = first, p_k = 0;
  bool p_prev_done = false;
  auto issue = [&](uint64_t k, uint64_t item, bool is_prev) {
    const int strip = (int)(item / n);
    const uint64_t j = item % n;
    const int y0 = strip * kRH;
    const int r0 = max(0, y0 - 2), r1 = min(H, y0 + kRH + 2);
    const uint8_t* tok;
    if (!is_prev) tok = slot_ptr(a.cur, pl.rd_cur0 + j);
    else if (a.dedup && j >= 1) tok = slot_ptr(a.cur, pl.rd_cur0 + j - 1);
    else tok = slot_ptr(a.prev, pl.rd_prev0 + j);
    uint8_t* dst = stages + (k % kStages) * stage_bytes + (size_t)(r0 - (y0 - 2)) * W;
    const uint32_t bytes = (uint32_t)(r1 - r0) * W;
    uint64_t* bar = &bars[k % kStages];
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(dst, tok + (size_t)r0 * W, bytes, bar);
  };

  uint64_t c_k = 0;     // index of the next load to be consumed
  for (uint64_t item = first; item < last; ++item) {
    const int strip = (int)(item / n);
    const uint64_t j = item % n;
    const uint64_t k_cur = c_k + (needs_prev_load(item) ? 1 : 0);
    if (threadIdx.x == 0) {
      const uint64_t limit = k_cur - 1 + kStages;
      while (p_k < limit && p_item < last) {
        if (needs_prev_load(p_item) && !p_prev_done) {
          issue(p_k, p_item, true);
          p_prev_done = true;
        } else {
          issue(p_k, p_item, false);
          ++p_item;
          p_prev_done = false;
        }
        ++p_k;
      }
      const uint64_t kp = k_cur - 1;
      const bool ok =
          mbar_wait_bounded(&bars[kp % kStages], (uint32_t)((kp / kStages) & 1), a.wait_limit_ns) &&
          mbar_wait_bounded(&bars[k_cur % kStages], (uint32_t)((k_cur / kStages) & 1),
                            a.wait_limit_ns);
      if (!ok) {
        s_abort = 1;
        set_status(a.eng, DF_ETIMEOUT, kWhereMdPipe);
      }
    }
    __syncthreads();
    if (s_abort) break;
    const uint8_t* cb = stages + (k_cur % kStages) * stage_bytes;
    const uint8_t* pb = stages + ((k_cur - 1) % kStages) * stage_bytes;
    const int y0 = strip * kRH;

    // 1. motion bits for buffer rows 0..kBufRows-1 (frame rows y0-2 .. y0+kRH+1);
    //    rows outside the frame read as all ones (erosion border).
    const int n_chunks = kBufRows * chunks_row;
    for (int base = 0; base < n_chunks; base += kMdThreads) {
      const int c = base + threadIdx.x;
      uint32_t half = 0;
      int row = 0, ch = 0;
      if (c < n_chunks) {
        row = c / chunks_row;
        ch = c - row * chunks_row;
        const int y = y0 - 2 + row;
        if (y < 0 || y >= H) {
          half = 0xffffu;
        } else {
          const size_t off = (size_t)row * W + ch * 16;
          half = motion_bits16(*reinterpret_cast<const uint4*>(cb + off),
                               *reinterpret_cast<const uint4*>(pb + off), thr4);
        }
      }
      const uint32_t other = __shfl_xor_sync(0xffffffffu, half, 1);
      if (c < n_chunks && !(threadIdx.x & 1)) bw[row * words + (ch >> 1)] = half | (other << 16);
    }
    __syncthreads();

    // 2. erosion for buffer rows 1..kBufRows-2; rows outside the frame become 0
    //    (dilation border).
    for (int e = threadIdx.x; e < (kBufRows - 2) * words; e += kMdThreads) {
      const int r = 1 + e / words, w = e % words;
      const int y = y0 - 2 + r;
      uint32_t v = 0;
      if (y >= 0 && y < H) {
        v = 0xffffffffu;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
          const uint32_t* row = bw + (r + dr) * words;
          const uint32_t b = row[w];
          const uint32_t l = w > 0 ? row[w - 1] >> 31 : 1u;
          const uint32_t rt = w < words - 1 ? row[w + 1] & 1u : 1u;
          v &= b & ((b << 1) | l) & ((b >> 1) | (rt << 31));
        }
      }
      ew[r * words + w] = v;
    }
    __syncthreads();

    // 3. dilation for the kRH strip rows, popcount of each 16-pixel half word.
    for (int e = threadIdx.x; e < kRH * words; e += kMdThreads) {
      const int r = 2 + e / words, w = e % words;
      const int y = y0 - 2 + r;
      uint32_t packed = 0;
      if (y < H) {
        uint32_t o = 0;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
          const uint32_t* row = ew + (r + dr) * words;
          const uint32_t v = row[w];
          const uint32_t l = w > 0 ? row[w - 1] >> 31 : 0u;
          const uint32_t rt = w < words - 1 ? row[w + 1] & 1u : 0u;
          o |= v | ((v << 1) | l) | ((v >> 1) | (rt << 31));
        }
        packed = (uint32_t)__popc(o & 0xffffu) | ((uint32_t)__popc(o >> 16) << 16);
      }
      pc[(r - 2) * words + w] = packed;
    }
    __syncthreads();

    // 4. tile counts of this strip (one tile row) and the frame's record total.
    int nz = 0;
    for (int base = 0; base < a.tiles_x; base += kMdThreads) {
      const int t = base + threadIdx.x;
      uint32_t cnt = 0;
      if (t < a.tiles_x) {
        const int w = t >> 1, sh = (t & 1) * 16;
        for (int r = 0; r < kRH; ++r) cnt += (pc[r * words + w] >> sh) & 0xffffu;
        a.counts[j * a.n_tiles + (size_t)strip * a.tiles_x + t] = (uint16_t)cnt;
      }
      nz += __syncthreads_count(cnt > 0);
    }
    if (threadIdx.x == 0 && nz) atomicAdd(&a.frame_tot[j], (uint32_t)nz);
    c_k = k_cur + 1;
    __syncthreads();
  }
  if (s_abort && threadIdx.x == 0) {
    // let copies still in flight land before the CTA's shared memory goes away
    for (uint64_t k = c_k; k < p_k; ++k)
      mbar_wait_bounded(&bars[k % kStages], (uint32_t)((k / kStages) & 1), a.wait_limit_ns);
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

cudaError_t launch_md_step(const MdArgs& a, int n_sm, cudaStream_t s) {
  const size_t smem = md_smem_bytes(a.W);
  cudaError_t e = cudaFuncSetAttribute(k_md_main, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_md_plan<<<1, 256, 0, s>>>(a);
  k_md_main<<<n_sm, kMdThreads, smem, s>>>(a);
  k_md_finish<<<1, 256, 0, s>>>(a);
  k_md_scatter<<<a.n_max, kMdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dfg
