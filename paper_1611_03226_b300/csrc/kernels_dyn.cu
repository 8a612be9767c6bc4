// Launchers of the bitmask-controlled dynamic actors (Poly, Adder).
#include "dyn_dev.cuh"

namespace dfg {

__global__ void k_dyn_plan(DynArgs a) { dyn_plan_dev(a); }
__global__ void k_poly_body(DynArgs a) { poly_body_dev(a, Grid{blockIdx.x, gridDim.x}); }
__global__ void k_add_body(DynArgs a) { add_body_dev(a, Grid{blockIdx.x, gridDim.x}); }

cudaError_t launch_dyn(const DynArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  k_dyn_plan<<<1, 256, 0, s>>>(a);
  if (ev0) cudaEventRecord(ev0, s);
  if (a.kind == DF_DPD_POLY) k_poly_body<<<n_sm * 8, 256, 0, s>>>(a);
  else k_add_body<<<n_sm * 8, 256, 0, s>>>(a);
  if (ev1) cudaEventRecord(ev1, s);
  return cudaGetLastError();
}

}  // namespace dfg
