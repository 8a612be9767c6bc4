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

// Publish the counters of a finished step (every body of the step has
// completed once griddep_wait returns).  This kernel, the spill kernel and the
// copy actor's kernels are launched as programmatic dependents: each waits for
// its predecessor before touching anything it wrote, so its launch overlaps
// the predecessor's end.
__global__ void k_publish(const EngineDev* e) {
  griddep_wait();
  if (!e->pub) return;
  for (uint32_t i = threadIdx.x; i < e->n_words; i += blockDim.x) e->pub[i] = e->ctr[i];
}

cudaError_t launch_publish(EngineDev* e, cudaStream_t s) {
  return launch_k(true, k_publish, dim3(1), dim3(256), 0, s, (const EngineDev*)e);
}

__global__ void k_spill(SpillArgs a) {
  griddep_wait();
  spill_dev(a, Grid{blockIdx.x, gridDim.x});
}

cudaError_t launch_spill(const SpillArgs& a, cudaStream_t s) {
  const uint64_t units = a.tok / a.unit;
  const unsigned blocks = (unsigned)std::min<uint64_t>(64, (units + 255) / 256);
  return launch_k(true, k_spill, dim3(blocks ? blocks : 1), dim3(256), 0, s, a);
}

__global__ void k_copy_plan(CopyArgs a) {
  griddep_wait();
  griddep_launch();
  copy_plan_dev(a);
}
__global__ void k_copy_body(CopyArgs a) {
  griddep_wait();
  copy_body_dev(a, Grid{blockIdx.x, gridDim.x});
}

cudaError_t launch_copy(const CopyArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1) {
  // timing events between the two kernels end the overlap, so none is asked for then
  const bool pdl = !ev0 && !ev1;
  cudaError_t e = launch_k(pdl, k_copy_plan, dim3(1), dim3(1), 0, s, a);
  if (e != cudaSuccess) return e;
  if (ev0) cudaEventRecord(ev0, s);
  e = launch_k(pdl, k_copy_body, dim3(n_sm * 4), dim3(256), 0, s, a);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, s);
  return cudaSuccess;
}

}  // namespace dfg
