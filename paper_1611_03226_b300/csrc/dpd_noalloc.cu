// Predistorter adjoint that never allocates device memory.
//
// df_dpd_backward keeps its tap-gradient partial sums in a buffer the library
// allocates with cudaMalloc (one per device and stream, grown on demand).  Some callers
// cannot let a library do that: a real-time adaptation loop (for example a
// radio front end refitting its predistorter between bursts) must not call
// cudaMalloc, which may synchronise the device and block for an unbounded
// time, and some host runtimes give a component a fixed device-memory budget
// with no new allocations after start-up.  This entry point runs the same
// kernels with the partial sums in a fixed array that is part of the loaded
// library image instead.
//
// The array is a file-scope __device__ variable.  In host code its name only
// stands in for the device object, so its device address is fetched with
// cudaGetSymbolAddress, with the calling device current, and passed to the
// kernels.  The lookup is repeated on every call (it is not a stream
// operation and costs far less than the kernels): an address cached across
// calls would go stale if the caller reset the device and the library's
// device code were loaded again.
#include "common.cuh"

namespace {

// Capacity of the fixed scratch: complex partial sums (1 MiB).
constexpr size_t kNoAllocScratchElems = 131072;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratchElems];

// Device address of the scratch array on the current device.
cudaError_t scratch_on_current_device(float2** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<float2*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" df_status df_dpd_backward_noalloc(const void* x, uint64_t n, const void* h, int32_t K,
                                             int32_t M, const int32_t* orders, const void* grad_y,
                                             void* grad_x, void* grad_h, void* cuda_stream) {
  if (((!x || !grad_y) && n) || !grad_h) return DF_EINVAL;
  if (!h || !orders || K < 1 || K > DF_MAX_BRANCHES || M < 1 || M > DF_MAX_TAPS) return DF_EINVAL;
  for (int k = 0; k < K; ++k)
    if (orders[k] < 1 || orders[k] % 2 == 0 || orders[k] > 63) return DF_EINVAL;
  if (dfg::dpd_backward_scratch_elems(n, K, M) > kNoAllocScratchElems) return DF_ENOTSUP;
  float2* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return DF_ECUDA;
  // Each call overwrites every partial sum it later reads, so nothing has to
  // be cleared between calls.
  const cudaError_t e = dfg::dpd_backward_stateless(
      static_cast<const float2*>(x), n, static_cast<const float2*>(h), K, M, orders,
      static_cast<const float2*>(grad_y), static_cast<float2*>(grad_x),
      static_cast<float2*>(grad_h), scratch, kNoAllocScratchElems,
      static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? DF_OK : DF_ECUDA;
}
