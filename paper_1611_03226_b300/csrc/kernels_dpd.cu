// Launchers of the fused predistortion actor (plan and body kernels).
#include <algorithm>
#include "dpd_dev.cuh"

namespace dfg {
// Padded tap count of the kernel instantiation for M taps (the padding taps
// are zero).  Between 8 and 16 an odd count takes the next even one: fewer
// code variants when actors of many tap counts share a launch, for one zero
// tap.
int dpd_supported_mt(int M) {
  if (M < 1 || M > 32) return 0;
  if (M <= 4) return 4;
  if (M <= 8) return 8;
  if (M <= 16) return (M + 1) & ~1;
  return 32;
}


// Both kernels may be launched as programmatic dependents (griddep_wait
// before touching anything an earlier kernel wrote); the plan lets the body
// launch at once, so the body's launch overlaps the plan.
__global__ void __launch_bounds__(256) k_dpd_plan(const DpdArgs* args) {
  griddep_wait();
  griddep_launch();
  dpd_plan_dev(args[blockIdx.x]);
}

// R = 8: two 256-thread CTAs per SM (128 registers); R = 16 holds twice the
// accumulators and may use more registers (one 256-thread CTA per SM, which is
// also what its shared memory allows).
template <int R, int MTMAX>
__global__ void __launch_bounds__(256, R == 8 ? 2 : 1) k_dpd_body(const DpdArgs* __restrict__ args,
                                                                   const uint16_t* __restrict__ order, int G) {
  extern __shared__ float4 smem_raw[];
  griddep_wait();
  dpd_body_dev<R, MTMAX>(args, order, G, Grid{blockIdx.x, gridDim.x}, smem_raw);
}

cudaError_t launch_dpd_plan(const DpdArgs* args_dev, int n_actors, cudaStream_t s, bool pdl) {
  if (n_actors <= 0) return cudaSuccess;
  return launch_k(pdl, k_dpd_plan, dim3(n_actors), dim3(256), 0, s, args_dev);
}

static size_t body_smem(int R, int mtmax, int warps, int G) {
  if (R == 8) return mtmax == 16 ? dpd_body_smem<8, 16>(warps, G) : dpd_body_smem<8, 32>(warps, G);
  return mtmax == 16 ? dpd_body_smem<16, 16>(warps, G) : dpd_body_smem<16, 32>(warps, G);
}

constexpr int kBodySmemMax = 226 * 1024;   // 227 KB per block less the static shared memory

template <int R, int MTMAX>
static cudaError_t body_attr() {
  return cudaFuncSetAttribute(k_dpd_body<R, MTMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kBodySmemMax);
}

cudaError_t dpd_prepare() {
  cudaError_t e;
  if ((e = body_attr<8, 16>()) != cudaSuccess) return e;
  if ((e = body_attr<8, 32>()) != cudaSuccess) return e;
  if ((e = body_attr<16, 16>()) != cudaSuccess) return e;
  return body_attr<16, 32>();
}

template <int R, int MTMAX>
static cudaError_t body_launch(const DpdArgs* args_dev, const uint16_t* order, int n_actors, uint32_t threads,
                               size_t smem, int n_sm, cudaStream_t s, bool pdl) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dpd_body<R, MTMAX>, threads, smem);
  return launch_k(pdl, k_dpd_body<R, MTMAX>, dim3(n_sm * std::max(per_sm, 1)), dim3(threads), smem, s,
                  args_dev, order, n_actors);
}

// tile = threads * R samples: every warp of the CTA takes chunks of 32 * R
// outputs (R = 8 or 16); threads = 32 .. 256.
cudaError_t launch_dpd_body(const DpdArgs* args_dev, const uint16_t* order, int n_actors, uint32_t tile,
                            uint32_t threads, int max_mt, int n_sm, cudaStream_t s, bool pdl) {
  if (n_actors <= 0) return cudaSuccess;
  if (n_actors > kMaxGroup || threads < 32 || threads > 256 || threads % 32) return cudaErrorInvalidValue;
  const int R = (int)(tile / threads);
  if ((R != 8 && R != 16) || tile != (uint32_t)R * threads) return cudaErrorInvalidValue;
  const int mtmax = max_mt <= 16 ? 16 : 32;
  const size_t smem = body_smem(R, mtmax, (int)threads / 32, n_actors);
  if (smem > (size_t)kBodySmemMax) return cudaErrorInvalidValue;
  if (R == 8) {
    return mtmax == 16 ? body_launch<8, 16>(args_dev, order, n_actors, threads, smem, n_sm, s, pdl)
                       : body_launch<8, 32>(args_dev, order, n_actors, threads, smem, n_sm, s, pdl);
  }
  return mtmax == 16 ? body_launch<16, 16>(args_dev, order, n_actors, threads, smem, n_sm, s, pdl)
                     : body_launch<16, 32>(args_dev, order, n_actors, threads, smem, n_sm, s, pdl);
}

}  // namespace dfg
