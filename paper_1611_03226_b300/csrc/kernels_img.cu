// Launchers of the image actors of the paper's motion pipeline (Sec. 4.1).
#include <algorithm>
#include "img_dev.cuh"

namespace dfg {

// The plan and the body are launched as programmatic dependents: each waits
// (griddep_wait) for its predecessor before touching anything it writes, and
// the plan lets the body launch at once, so the body's launch overlaps the plan.
__global__ void k_img_plan(const __grid_constant__ ImgArgs a) {
  griddep_wait();
  griddep_launch();
  if (threadIdx.x == 0) img_plan_dev(a);
}

// One body kernel per actor kind, so that each gets the registers it needs.
template <int KIND>
__global__ void __launch_bounds__(kImgThreads) k_img_body(const __grid_constant__ ImgArgs a) {
  extern __shared__ float4 img_smem[];
  __shared__ ImgPlan s_pl;
  griddep_wait();
  if (threadIdx.x == 0) s_pl = *a.plan;
  __syncthreads();
  if (s_pl.n == 0) return;
  const Grid g{blockIdx.x, gridDim.x};
  if constexpr (KIND == DF_THRES) thres_body(a, s_pl, g);
  else if constexpr (KIND == DF_GAUSS5) gauss_body(a, s_pl, g, reinterpret_cast<uint8_t*>(img_smem));
  else med_body(a, s_pl, g, reinterpret_cast<uint8_t*>(img_smem));
}

static int g_img_blocks_per_sm[3] = {0, 0, 0};

template <int KIND>
static cudaError_t prepare_one(int slot) {
  const size_t smem = KIND == DF_THRES ? 0 : img_smem_bytes(kImgMaxWidth);
  cudaError_t e = cudaFuncSetAttribute(k_img_body<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_img_body<KIND>, kImgThreads,
                                                    KIND == DF_THRES ? 0 : img_smem_bytes(320));
  if (e != cudaSuccess) return e;
  g_img_blocks_per_sm[slot] = std::max(per_sm, 1);
  return cudaSuccess;
}

cudaError_t img_prepare() {
  if (g_img_blocks_per_sm[0]) return cudaSuccess;
  cudaError_t e = prepare_one<DF_GAUSS5>(0);
  if (e == cudaSuccess) e = prepare_one<DF_THRES>(1);
  if (e == cudaSuccess) e = prepare_one<DF_MED5>(2);
  return e;
}

cudaError_t launch_img(const ImgArgs& a, int n_sm, cudaStream_t s) {
  cudaError_t e = launch_k(true, k_img_plan, dim3(1), dim3(32), 0, s, a);
  if (e != cudaSuccess) return e;
  const int slot = a.kind == DF_GAUSS5 ? 0 : (a.kind == DF_THRES ? 1 : 2);
  const dim3 grid(n_sm * std::max(g_img_blocks_per_sm[slot], 1));
  const size_t smem = a.kind == DF_THRES ? 0 : img_smem_bytes(a.W);
  if (a.kind == DF_GAUSS5) return launch_k(true, k_img_body<DF_GAUSS5>, grid, dim3(kImgThreads), smem, s, a);
  if (a.kind == DF_THRES) return launch_k(true, k_img_body<DF_THRES>, grid, dim3(kImgThreads), smem, s, a);
  return launch_k(true, k_img_body<DF_MED5>, grid, dim3(kImgThreads), smem, s, a);
}

}  // namespace dfg
