// Launchers of the image actors of the paper's motion pipeline (Sec. 4.1).
#include <algorithm>
#include "img_dev.cuh"

namespace dfg {

__global__ void k_img_plan(const __grid_constant__ ImgArgs a) {
  if (threadIdx.x == 0) img_plan_dev(a);
}

__global__ void __launch_bounds__(kImgThreads) k_img_body(const __grid_constant__ ImgArgs a) {
  extern __shared__ float4 img_smem[];
  img_body_dev(a, Grid{blockIdx.x, gridDim.x}, reinterpret_cast<uint8_t*>(img_smem));
}

static int g_img_blocks_per_sm = 0;

cudaError_t img_prepare() {
  if (g_img_blocks_per_sm) return cudaSuccess;
  const size_t smem = img_smem_bytes(kImgMaxWidth);
  cudaError_t e = cudaFuncSetAttribute(k_img_body, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_img_body, kImgThreads, img_smem_bytes(320));
  if (e != cudaSuccess) return e;
  g_img_blocks_per_sm = std::max(per_sm, 1);
  return cudaSuccess;
}

cudaError_t launch_img(const ImgArgs& a, int n_sm, cudaStream_t s) {
  k_img_plan<<<1, 32, 0, s>>>(a);
  const size_t smem = a.kind == DF_THRES ? 0 : img_smem_bytes(a.W);
  k_img_body<<<n_sm * std::max(g_img_blocks_per_sm, 1), kImgThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dfg
