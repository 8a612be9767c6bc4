// Persistent step kernel: one cooperative launch runs n steps of the whole
// program (or steps until one fires nothing), with every rate decision, scan,
// gather and scatter on the device and no host involvement between steps.
//
// Phases of one step follow the per-phase kernels exactly (plan -> body ->
// finish -> scatter per actor, actors in insertion order); a grid barrier
// separates phases that consume another CTA's results.  The barrier is one
// 64-bit arrival count in the engine state (each CTA adds 1 with release
// semantics and polls it with acquire loads), so no CTA has to learn that it
// arrived last before the others may go on.  An error anywhere adds
// kBarrierError to the count: every waiting CTA sees it in the word it polls
// and leaves, and a CTA that waits longer than the limit records DF_ETIMEOUT
// (which adds it), so a wait that cannot complete ends the kernel instead of
// hanging it, after about one wait limit.
#include "core_dev.cuh"
#include "dpd_dev.cuh"
#include "dyn_dev.cuh"
#include "md_dev.cuh"
#include "img_dev.cuh"

namespace dfg {

__device__ __forceinline__ long long timer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Copy of the counters for concurrent host I/O once a step is over.
__device__ void publish_counters(EngineDev* e) {
  if (e->pub)
    for (uint32_t i = 0; i < e->n_words; ++i) e->pub[i] = reinterpret_cast<volatile uint64_t*>(e->ctr)[i];
}

// The barriers of one launch.  bar_arrive is a multiple of the grid size nb
// whenever no CTA of a launch is inside a barrier (the count starts at 0 and
// every barrier adds nb); when a launch starts, CTAs of the same launch may
// already have arrived at its first barrier, never all of them, so each CTA
// rounds what it reads down to a multiple of nb to find where the launch
// began.  Barrier b (0-based) of the launch completes at base + (b + 1) nb.
// (The grid size of a network's launches never changes; the wait self-test
// uses its own grid and clears the count before and after.)
struct GridBarrier {
  unsigned long long target;   // valid in thread 0
  unsigned int nb;
  bool ok;                     // false: an error was recorded; leave
};

__device__ GridBarrier grid_barrier_begin(EngineDev* e, unsigned int nb) {
  __shared__ unsigned long long s_v;
  if (threadIdx.x == 0) s_v = ld_acquire_u64(&e->bar_arrive);
  __syncthreads();
  const unsigned long long v = s_v;
  GridBarrier g;
  g.nb = nb;
  g.ok = v < kBarrierError;
  g.target = v - v % nb;
  __syncthreads();
  return g;
}

// Returns false when an error was recorded (own timeout or any other).
__device__ bool grid_barrier(EngineDev* e, GridBarrier& g, long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    g.target += g.nb;
    red_release_add_u64(&e->bar_arrive, 1ull);
    unsigned long long v;
    unsigned int polls = 0;
    long long t0 = 0;
    while ((v = ld_acquire_u64(&e->bar_arrive)) < g.target) {
      // a short pause between polls: hundreds of CTAs polling one word back to
      // back slow the memory accesses of the CTAs still working (measured on
      // a one-actor step: its plan ran 0.6 us faster)
      __nanosleep(256);
      if ((++polls & 63u) == 0) {
        const long long t = timer_ns();
        if (t0 == 0) {
          t0 = t;
        } else if (t - t0 > limit_ns) {
          set_status(e, DF_ETIMEOUT, kWhereGridBarrier);
          v = kBarrierError;
          break;
        }
      }
    }
    s_ok = v < kBarrierError;
  }
  __syncthreads();
  g.ok = s_ok != 0;
  return g.ok;
}

__device__ __forceinline__ unsigned long long fired_now(EngineDev* e) {
  return *reinterpret_cast<volatile unsigned long long*>(&e->fired_total);
}

// Each phase is its own call, so that its registers are allocated for it
// alone and a phase that needs many does not make the others spill.
__device__ __noinline__ void ph_copy_body(const CopyArgs& a, Grid g) { copy_body_dev(a, g); }
__device__ __noinline__ void ph_dpd_plan(const DpdArgs* args, int n) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    dpd_plan_dev(args[i]);
    __syncthreads();
  }
}
template <int MTMAX>
__device__ __noinline__ void ph_dpd_body(const DpdArgs* args, const uint16_t* order, int n, Grid g, float4* smem) {
  dpd_body_dev<8, MTMAX>(args, order, n, g, smem);
}
__device__ __noinline__ void ph_dyn_body(const DynArgs& a, Grid g) {
  if (a.kind == DF_DPD_POLY) poly_body_dev(a, g);
  else add_body_dev(a, g);
}
__device__ __noinline__ void ph_img_body(const ImgArgs& a, Grid g, uint8_t* smem) { img_body_dev(a, g, smem); }
__device__ __noinline__ void ph_md_main(const MdArgs& a, Grid g) {
  if (a.shared_rows) md_main_dev<8, false>(a, g);
  else md_main_dev<2, false>(a, g);
}
__device__ __noinline__ void ph_md_emit(const MdArgs& a, Grid g) { md_emit_dev(a, g); }

template <int MTMAX>
__global__ void __launch_bounds__(kPersistThreads, 2) k_persistent(const PersistOp* __restrict__ ops,
                                                               int n_ops, EngineDev* eng,
                                                               int64_t n_steps, long long limit_ns,
                                                               bool publish) {
  extern __shared__ float4 smem[];
  const Grid g{blockIdx.x, gridDim.x};
  const bool lead = blockIdx.x == 0;
  const int64_t max_steps = n_steps < 0 ? (int64_t)1 << 20 : n_steps;
  const bool until_quiet = n_steps < 0;
  if (n_ops == 0) return;
  // An error recorded by an earlier launch stays until the host clears it
  // (with the barrier count): nothing runs on top of it.
  GridBarrier gb = grid_barrier_begin(eng, gridDim.x);
  if (!gb.ok) return;
  unsigned long long fired0 = 0;
  if (until_quiet) {
    // the firing total before any commit: no plan runs before this barrier
    fired0 = fired_now(eng);
    if (!grid_barrier(eng, gb, limit_ns)) return;
  }
  for (int64_t step = 0; step < max_steps; ++step) {
    unsigned long long fired1 = 0;
    for (int o = 0; o < n_ops; ++o) {
      const PersistOp op = ops[o];
      if (op.kind == kPersistCopy) {
        const CopyArgs& a = *static_cast<const CopyArgs*>(op.args);
        if (lead && threadIdx.x == 0) copy_plan_dev(a);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_copy_body(a, g);
      } else if (op.kind == kPersistDpd) {
        const DpdArgs* args = static_cast<const DpdArgs*>(op.args);
        ph_dpd_plan(args, op.n);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_dpd_body<MTMAX>(args, op.order, op.n, g, smem);
      } else if (op.kind == kPersistDyn) {
        const DynArgs& a = *static_cast<const DynArgs*>(op.args);
        if (lead) dyn_plan_dev(a);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_dyn_body(a, g);
      } else if (op.kind == kPersistImg) {
        const ImgArgs& a = *static_cast<const ImgArgs*>(op.args);
        if (lead && threadIdx.x == 0) img_plan_dev(a);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_img_body(a, g, reinterpret_cast<uint8_t*>(smem));
      } else if (op.kind == kPersistSpill) {
        // the writer op before this one ended with a barrier: its tokens are in place
        const SpillArgs* sp = static_cast<const SpillArgs*>(op.args);
        for (int i = 0; i < op.n; ++i) spill_dev(sp[i], g);
      } else if (op.kind == kPersistMd) {
        const MdArgs& a = *static_cast<const MdArgs*>(op.args);
        if (lead) md_plan_dev(a);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_md_main(a, g);
        if (!grid_barrier(eng, gb, limit_ns)) return;
        ph_md_emit(a, g);
      }
      // after the last fixed step the end of the kernel orders what follows
      if (!until_quiet && o == n_ops - 1 && step == max_steps - 1) break;
      // Every plan of the step has committed (each was followed by a barrier
      // this CTA passed) and none of the next step can start before this
      // barrier completes, so every CTA reads the same step total here.
      if (o == n_ops - 1 && until_quiet) fired1 = fired_now(eng);
      if (!grid_barrier(eng, gb, limit_ns)) return;
      if (o == n_ops - 1 && publish) {
        // the step's bodies are done: publish its counters for concurrent
        // host I/O before any plan of the next step commits
        if (lead && threadIdx.x == 0) publish_counters(eng);
        if (!grid_barrier(eng, gb, limit_ns)) return;
      }
    }
    if (until_quiet) {
      if (fired1 == fired0) return;
      fired0 = fired1;
    }
  }
  // fixed step count: with concurrent host I/O the last CTA to finish
  // publishes the counters (and returns exit_count to 0 for the next launch)
  if (!publish) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&eng->exit_count, 1u) == gridDim.x - 1) {
      __threadfence();
      publish_counters(eng);
      eng->exit_count = 0;
    }
  }
}

// A barrier that waits for one more CTA than the grid has: it can only end by
// its time limit, which must leave DF_ETIMEOUT in the status word.
__global__ void k_barrier_selftest(EngineDev* eng, long long limit_ns) {
  GridBarrier gb = grid_barrier_begin(eng, gridDim.x + 1);
  if (gb.ok) grid_barrier(eng, gb, limit_ns);
}

static int g_persist_blocks[2] = {0, 0};

cudaError_t persistent_prepare(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_persistent<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_persistent<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_persist_blocks[0], k_persistent<16>,
                                                    kPersistThreads, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_persist_blocks[1], k_persistent<32>,
                                                       kPersistThreads, smem);
}

size_t persistent_smem(int mtmax, int max_group) {
  return mtmax <= 16 ? dpd_body_smem<8, 16>(kPersistThreads / 32, max_group)
                     : dpd_body_smem<8, 32>(kPersistThreads / 32, max_group);
}

// The barrier count is a multiple of the grid size, and exit_count 0, when
// the engine is created and after every launch that ends without an error; an
// error leaves kBarrierError in the count, which later launches check first,
// and whoever clears the status word clears the barrier state with it.
cudaError_t launch_persistent(const PersistOp* ops, int n_ops, EngineDev* eng, int64_t n_steps,
                              long long limit_ns, int mtmax, size_t smem, int n_sm, int per_sm_cap,
                              bool publish, cudaStream_t s) {
  const int idx = mtmax <= 16 ? 0 : 1;
  const int per_sm = per_sm_cap > 0 ? std::min(per_sm_cap, g_persist_blocks[idx]) : g_persist_blocks[idx];
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // a cooperative launch (all CTAs resident at once), also inside a CUDA graph capture
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(n_sm * per_sm);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (idx == 0) return cudaLaunchKernelEx(&cfg, k_persistent<16>, ops, n_ops, eng, n_steps, limit_ns, publish);
  return cudaLaunchKernelEx(&cfg, k_persistent<32>, ops, n_ops, eng, n_steps, limit_ns, publish);
}

cudaError_t launch_barrier_selftest(EngineDev* eng, long long limit_ns, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&eng->bar_arrive, 0, sizeof(unsigned long long) + sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&eng, (void*)&limit_ns};
  return cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(4), dim3(32), args, 0, s);
}

}  // namespace dfg
