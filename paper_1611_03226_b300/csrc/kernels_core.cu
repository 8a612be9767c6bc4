// Counter maintenance and the launchers of the copy actor.
#include <algorithm>

#include "core_dev.cuh"

namespace dfg {

__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }
__global__ void k_add_u64(uint64_t* p, uint64_t v) { *p += v; }

cudaError_t launch_set_u64(uint64_t* p, uint64_t v, cudaStream_t s) {
  k_set_u64<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}
cudaError_t launch_add_u64(uint64_t* p, uint64_t v, cudaStream_t s) {
  k_add_u64<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

// Publish the counters of a finished step (stream order: every body of the
// step has completed when this runs).
__global__ void k_publish(const EngineDev* e) {
  if (!e->pub) return;
  for (uint32_t i = threadIdx.x; i < e->n_words; i += blockDim.x) e->pub[i] = e->ctr[i];
}

cudaError_t launch_publish(EngineDev* e, cudaStream_t s) {
  k_publish<<<1, 256, 0, s>>>(e);
  return cudaGetLastError();
}

__global__ void k_spill(SpillArgs a) { spill_dev(a, Grid{blockIdx.x, gridDim.x}); }

cudaError_t launch_spill(const SpillArgs& a, cudaStream_t s) {
  const uint64_t units = a.tok / a.unit;
  const unsigned blocks = (unsigned)std::min<uint64_t>(64, (units + 255) / 256);
  k_spill<<<blocks ? blocks : 1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

__global__ void k_copy_plan(CopyArgs a) { copy_plan_dev(a); }
__global__ void k_copy_body(CopyArgs a) { copy_body_dev(a, Grid{blockIdx.x, gridDim.x}); }

cudaError_t launch_copy(const CopyArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1) {
  k_copy_plan<<<1, 1, 0, s>>>(a);
  if (ev0) cudaEventRecord(ev0, s);
  k_copy_body<<<n_sm * 4, 256, 0, s>>>(a);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

}  // namespace dfg
