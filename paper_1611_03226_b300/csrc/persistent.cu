// Persistent step kernel: one cooperative launch runs n steps of the whole
// program (or steps until one fires nothing), with every rate decision, scan,
// gather and scatter on the device and no host involvement between steps.
//
// Phases of one step follow the per-phase kernels exactly (plan -> body ->
// finish -> scatter per actor, actors in insertion order); a grid barrier
// separates phases that consume another CTA's results.  The barrier is a
// counter plus a generation word in the engine state; a CTA that waits longer
// than the limit records DF_ETIMEOUT in the status word, and every CTA that is
// waiting, or reaches a barrier later, leaves as soon as it sees the status
// word set, so a wait that cannot complete ends the kernel instead of hanging
// it, after about one wait limit.
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

// Copy of the counters for concurrent host I/O once a step is over.
__device__ void publish_counters(EngineDev* e) {
  if (e->pub)
    for (uint32_t i = 0; i < e->n_words; ++i) e->pub[i] = reinterpret_cast<volatile uint64_t*>(e->ctr)[i];
}

// Returns false when the status word is set (own timeout or another CTA's).
// With snap, the CTA that releases the barrier records fired_total in
// total_snap first, so every CTA reads the same value after the barrier (a
// CTA that reads fired_total itself may already see the next phase's commits).
__device__ bool grid_barrier(EngineDev* e, unsigned int expected, long long limit_ns,
                             bool snap = false) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &e->barrier_gen;
    const unsigned int g0 = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&e->barrier_count, 1u) + 1u;
    int ok = 1;
    if (arrived == expected) {
      e->barrier_count = 0;
      if (snap) {
        e->total_snap = *reinterpret_cast<volatile unsigned long long*>(&e->fired_total);
        // the step is over: publish its counters for concurrent host I/O
        publish_counters(e);
      }
      __threadfence();
      atomicAdd(&e->barrier_gen, 1u);
    } else {
      const long long t0 = timer_ns();
      volatile int32_t* status = &e->status;
      while (*gen == g0) {
        // another CTA's timeout or error ends this wait at once
        if (*status != 0) {
          ok = 0;
          break;
        }
        if (timer_ns() - t0 > limit_ns) {
          set_status(e, DF_ETIMEOUT, kWhereGridBarrier);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && *reinterpret_cast<volatile int32_t*>(&e->status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

template <int MTMAX>
__global__ void __launch_bounds__(kPersistThreads, 2) k_persistent(const PersistOp* __restrict__ ops,
                                                               int n_ops, EngineDev* eng,
                                                               int64_t n_steps, long long limit_ns) {
  extern __shared__ float4 smem[];
  const Grid g{blockIdx.x, gridDim.x};
  const unsigned int nb = gridDim.x;
  const bool lead = blockIdx.x == 0;
  const int64_t max_steps = n_steps < 0 ? (int64_t)1 << 20 : n_steps;
  const bool until_quiet = n_steps < 0;
  volatile unsigned long long* snap = &eng->total_snap;
  if (n_ops == 0) return;
  unsigned long long fired0 = 0;
  if (until_quiet) {
    // the first barrier records the firing total before any commit
    if (!grid_barrier(eng, nb, limit_ns, true)) return;
    fired0 = *snap;
  }
  for (int64_t step = 0; step < max_steps; ++step) {
    for (int o = 0; o < n_ops; ++o) {
      const PersistOp op = ops[o];
      if (op.kind == kPersistCopy) {
        const CopyArgs& a = *static_cast<const CopyArgs*>(op.args);
        if (lead && threadIdx.x == 0) copy_plan_dev(a);
        if (!grid_barrier(eng, nb, limit_ns)) return;
        copy_body_dev(a, g);
      } else if (op.kind == kPersistDpd) {
        const DpdArgs* args = static_cast<const DpdArgs*>(op.args);
        for (int i = blockIdx.x; i < op.n; i += gridDim.x) {
          dpd_plan_dev(args[i]);
          __syncthreads();
        }
        if (!grid_barrier(eng, nb, limit_ns)) return;
        dpd_body_dev<8, MTMAX>(args, op.order, op.n, g, smem);
      } else if (op.kind == kPersistDyn) {
        const DynArgs& a = *static_cast<const DynArgs*>(op.args);
        if (lead) dyn_plan_dev(a);
        if (!grid_barrier(eng, nb, limit_ns)) return;
        if (a.kind == DF_DPD_POLY) poly_body_dev(a, g);
        else add_body_dev(a, g);
      } else if (op.kind == kPersistImg) {
        const ImgArgs& a = *static_cast<const ImgArgs*>(op.args);
        if (lead && threadIdx.x == 0) img_plan_dev(a);
        if (!grid_barrier(eng, nb, limit_ns)) return;
        img_body_dev(a, g, reinterpret_cast<uint8_t*>(smem));
      } else if (op.kind == kPersistSpill) {
        // the writer op before this one ended with a barrier: its tokens are in place
        const SpillArgs* sp = static_cast<const SpillArgs*>(op.args);
        for (int i = 0; i < op.n; ++i) spill_dev(sp[i], g);
      } else if (op.kind == kPersistMd) {
        const MdArgs& a = *static_cast<const MdArgs*>(op.args);
        if (lead) md_plan_dev(a);
        if (!grid_barrier(eng, nb, limit_ns)) return;
        if (a.shared_rows) md_main_dev<8, false>(a, g);
        else md_main_dev<2, false>(a, g);
        if (!grid_barrier(eng, nb, limit_ns)) return;
        md_emit_dev(a, g);
      }
      // the step's last barrier records the total that ends the step; after the
      // last step of a fixed count the end of the kernel orders what follows
      if (!until_quiet && o == n_ops - 1 && step == max_steps - 1) break;
      if (!grid_barrier(eng, nb, limit_ns, o == n_ops - 1)) return;
    }
    if (until_quiet) {
      // every CTA reads the same recorded total, so all take the same decision
      const unsigned long long fired1 = *snap;
      if (fired1 == fired0) return;
      fired0 = fired1;
    }
  }
  // fixed step count: the last CTA to finish publishes the counters
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&eng->exit_count, 1u) == nb - 1) {
      __threadfence();
      eng->total_snap = *reinterpret_cast<volatile unsigned long long*>(&eng->fired_total);
      publish_counters(eng);
    }
  }
}

// A barrier that waits for one more CTA than the grid has: it can only end by
// its time limit, which must leave DF_ETIMEOUT in the status word.
__global__ void k_barrier_selftest(EngineDev* eng, long long limit_ns) {
  grid_barrier(eng, gridDim.x + 1, limit_ns);
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

cudaError_t launch_persistent(const PersistOp* ops, int n_ops, EngineDev* eng, int64_t n_steps,
                              long long limit_ns, int mtmax, size_t smem, int n_sm, cudaStream_t s) {
  const int idx = mtmax <= 16 ? 0 : 1;
  const int per_sm = g_persist_blocks[idx];
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(&eng->barrier_count, 0, 3 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
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
  if (idx == 0) return cudaLaunchKernelEx(&cfg, k_persistent<16>, ops, n_ops, eng, n_steps, limit_ns);
  return cudaLaunchKernelEx(&cfg, k_persistent<32>, ops, n_ops, eng, n_steps, limit_ns);
}

cudaError_t launch_barrier_selftest(EngineDev* eng, long long limit_ns, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(&eng->barrier_count, 0, 3 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&eng, (void*)&limit_ns};
  return cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(4), dim3(32), args, 0, s);
}

}  // namespace dfg
