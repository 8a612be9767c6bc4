// Launchers of the fused motion-detection actor.
#include <algorithm>
#include "md_dev.cuh"

namespace dfg {

size_t md_smem_bytes(int W) {
  (void)W;
  return 0;
}

__global__ void k_md_plan(MdArgs a) { md_plan_dev(a); }

template <int F>
__global__ void __launch_bounds__(kMdWarpsPerCta * 32) k_md_main(MdArgs a) {
  md_main_dev<F, true>(a, Grid{blockIdx.x, gridDim.x});
}

__global__ void __launch_bounds__(kMdThreads) k_md_emit(MdArgs a) {
  const uint64_t n = a.plan->n_cand;
  if (blockIdx.x < (n > 0 ? n : 1)) md_emit_frame(a, blockIdx.x, blockIdx.x == 0);
}

static int g_md_blocks_per_sm[2] = {0, 0};

cudaError_t md_prepare(int W) {
  (void)W;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md_main<kMdFrames>,
                                                                kMdWarpsPerCta * 32, 0);
  if (e != cudaSuccess) return e;
  g_md_blocks_per_sm[0] = per_sm > 0 ? per_sm : 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_md_main<2>, kMdWarpsPerCta * 32, 0);
  if (e != cudaSuccess) return e;
  g_md_blocks_per_sm[1] = per_sm > 0 ? per_sm : 1;
  return cudaSuccess;
}

cudaError_t launch_md_step(const MdArgs& a, const MdTma* tma, int n_sm, cudaStream_t s,
                           cudaEvent_t ev0, cudaEvent_t ev1) {
  k_md_plan<<<1, 256, 0, s>>>(a);
  if (ev0) cudaEventRecord(ev0, s);
  if (tma && tma->ok)
    launch_md_main_tma(a, *tma, n_sm, s);
  else if (a.shared_rows)
    k_md_main<kMdFrames><<<n_sm * std::max(g_md_blocks_per_sm[0], 1), kMdWarpsPerCta * 32, 0, s>>>(a);
  else
    k_md_main<2><<<n_sm * std::max(g_md_blocks_per_sm[1], 1), kMdWarpsPerCta * 32, 0, s>>>(a);
  if (ev1) cudaEventRecord(ev1, s);
  k_md_emit<<<a.n_max, kMdThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dfg
