// Launchers of the fused motion-detection actor.
#include <algorithm>
#include "md_dev.cuh"

namespace dfg {

size_t md_smem_bytes(int W) {
  (void)W;
  return 0;
}

__global__ void k_md_plan(MdArgs a) {
  griddep_wait();
  griddep_launch();
  md_plan_dev(a);
}

template <int F>
__global__ void __launch_bounds__(kMdWarpsPerCta * 32) k_md_main(MdArgs a) {
  md_main_dev<F, true>(a, Grid{blockIdx.x, gridDim.x});
}

__global__ void __launch_bounds__(kMdThreads) k_md_emit(MdArgs a) {
  griddep_wait();
  md_emit_frame(a, blockIdx.x, blockIdx.x == 0);   // frames past the candidates return at once
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
  // Without timing events between them, the plan, main and emit kernels are
  // launched as programmatic dependents: each starts (and waits in
  // griddep_wait) while its predecessor finishes, which hides launch latency.
  const bool pdl = tma && tma->ok && !ev0 && !ev1;
  cudaError_t e = launch_k(pdl, k_md_plan, dim3(1), dim3(256), 0, s, a);
  if (e != cudaSuccess) return e;
  if (ev0) cudaEventRecord(ev0, s);
  if (tma && tma->ok)
    e = launch_md_main_tma(a, *tma, n_sm, s, pdl);
  else if (a.shared_rows)
    k_md_main<kMdFrames><<<n_sm * std::max(g_md_blocks_per_sm[0], 1), kMdWarpsPerCta * 32, 0, s>>>(a);
  else
    k_md_main<2><<<n_sm * std::max(g_md_blocks_per_sm[1], 1), kMdWarpsPerCta * 32, 0, s>>>(a);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, s);
  e = launch_k(pdl, k_md_emit, dim3(a.n_max), dim3(kMdThreads), 0, s, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dfg
