// Launchers of the fused predistortion actor and the stateless differentiable
// predistorter (forward and adjoint).
#include <algorithm>
#include "dpd_dev.cuh"

namespace dfg {
int dpd_supported_mt(int M) {
  if (M < 1 || M > 32) return 0;
  if (M <= 4) return 4;
  if (M <= 8) return 8;
  if (M <= 16) return M;
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

// ------------------------------------------------- stateless operators ----
// One signal, all branches active, zero history.  Taps arrive unpadded (K*M);
// they are read with padding on the fly: tap m >= M contributes zero.
constexpr int kStatelessR = 8;
constexpr int kStatelessP = 128;

struct StatelessArgs {
  const float2* x;
  const float2* gy;
  float2* y;            // forward output or grad_x
  float2* partial;      // [tiles][K][MT] tap-gradient partial sums
  float2* gh;           // [K][M]
  const float2* h;      // [K][M] taps
  uint64_t n;
  int K, M, MT;
  int orders[kMaxBranches];
};

template <int R, int MT>
__device__ void fwd_tile(const StatelessArgs& a, uint64_t tile, float2* xs, float2* zs) {
  const int P = blockDim.x, p = threadIdx.x;
  const uint64_t T = (uint64_t)R * P;
  const uint64_t t0 = tile * T;
  const int len = (int)min(T, a.n - t0);
  const int W = (int)T + MT - 1;
  for (int v = p; v < W; v += P) {
    const int64_t pos = (int64_t)t0 - (MT - 1) + v;
    xs[v] = (pos >= 0 && pos < (int64_t)(t0 + len)) ? a.x[pos] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int k = 0; k < a.K; ++k) {
    const int q = (a.orders[k] - 1) >> 1;
    for (int v = p; v < W; v += P) zs[v + v / R] = psi_q(xs[v], q);
    __syncthreads();
    fir_branch<R, MT>(acc, zs, p, a.h + (size_t)k * a.M, a.M);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) zs[p * (R + 1) + r] = acc[r];
  __syncthreads();
  for (int o = p; o < len; o += P) a.y[t0 + o] = zs[o + o / R];
  __syncthreads();
}

template <int R>
__global__ void __launch_bounds__(kStatelessP) k_dpd_fwd(StatelessArgs a) {
  extern __shared__ float4 smem_raw[];
  const uint64_t T = (uint64_t)R * blockDim.x;
  const uint64_t nt = (a.n + T - 1) / T;
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  float2* zs = xs + (T + a.MT);
  for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    switch (a.MT) {
#define FWD_CASE(MTV) case MTV: fwd_tile<R, MTV>(a, t, xs, zs); break;
      DPD_MT_CASES(FWD_CASE)
#undef FWD_CASE
      default: break;
    }
  }
}

// Deterministic block sum of one float2 per thread into out (thread 0 writes).
__device__ float2 block_sum_f2(float2 v, float2* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float2 s = make_float2(0.f, 0.f);
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) { s.x += red[w].x; s.y += red[w].y; }
  __syncthreads();
  return s;
}

template <int R, int MC>
__device__ void gh_reduce_chunk(const StatelessArgs& a, uint64_t tile, int k, int m0,
                                const float2 (&gr)[R], const float2* zs, int shift, float2* red) {
  float2 ph[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) ph[m] = make_float2(0.f, 0.f);
  gh_chunk<R, MC>(ph, gr, zs, threadIdx.x, shift);
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const float2 s = block_sum_f2(ph[m], red);
    if (threadIdx.x == 0) a.partial[(tile * a.K + k) * a.MT + m0 + m] = s;
  }
}

template <int R, int MT>
__device__ void bwd_tile(const StatelessArgs& a, uint64_t tile, float2* xs, float2* zs, float2* gs,
                         float2* red) {
  const int P = blockDim.x, p = threadIdx.x;
  const uint64_t T = (uint64_t)R * P;
  const uint64_t t0 = tile * T;
  const int len = (int)min(T, a.n - t0);
  const int W = (int)T + MT - 1;
  for (int v = p; v < W; v += P) {
    const int64_t pos = (int64_t)t0 - (MT - 1) + v;
    xs[v] = (pos >= 0 && pos < (int64_t)(t0 + len)) ? a.x[pos] : make_float2(0.f, 0.f);
    const uint64_t gp = t0 + v;       // g window [t0, t0 + T + MT - 1), zero beyond n
    gs[v + v / R] = gp < a.n ? a.gy[gp] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 gr[R], gx[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    gr[r] = (p * R + r < len) ? gs[p * (R + 1) + r] : make_float2(0.f, 0.f);
    gx[r] = make_float2(0.f, 0.f);
  }
  for (int k = 0; k < a.K; ++k) {
    const int q = (a.orders[k] - 1) >> 1;
    for (int v = p; v < W; v += P) zs[v + v / R] = psi_q(xs[v], q);
    __syncthreads();
    const float2* hk = a.h + (size_t)k * a.M;
    float2 gz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) gz[r] = make_float2(0.f, 0.f);
    if constexpr (MT <= 16) {
      gh_reduce_chunk<R, MT>(a, tile, k, 0, gr, zs, 0, red);
      fir_anticausal_conj<R, MT>(gz, gs, p, 0, hk, a.M);
    } else {
      gh_reduce_chunk<R, 16>(a, tile, k, 0, gr, zs, 16, red);
      gh_reduce_chunk<R, 16>(a, tile, k, 16, gr, zs, 0, red);
      fir_anticausal_conj<R, 16>(gz, gs, p, 0, hk, a.M);
      fir_anticausal_conj<R, 16>(gz, gs, p, 16, hk + 16, a.M - 16);
    }
    if (a.y) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 x = xs[p * R + r + MT - 1];
        const float u = fmaf(x.x, x.x, x.y * x.y);
        float uq1 = 1.f;
        for (int i = 0; i + 1 < q; ++i) uq1 *= u;
        const float uq = q > 0 ? uq1 * u : 1.f;
        const float c1 = (q + 1) * uq;
        gx[r].x = fmaf(c1, gz[r].x, gx[r].x);
        gx[r].y = fmaf(c1, gz[r].y, gx[r].y);
        if (q > 0) {
          const float c2 = q * uq1;
          const float2 x2 = make_float2(x.x * x.x - x.y * x.y, 2.f * x.x * x.y);
          // c2 * x^2 * conj(gz)
          gx[r].x = fmaf(c2, x2.x * gz[r].x + x2.y * gz[r].y, gx[r].x);
          gx[r].y = fmaf(c2, x2.y * gz[r].x - x2.x * gz[r].y, gx[r].y);
        }
      }
    }
    __syncthreads();
  }
  if (a.y) {
#pragma unroll
    for (int r = 0; r < R; ++r) zs[p * (R + 1) + r] = gx[r];
    __syncthreads();
    for (int o = p; o < len; o += P) a.y[t0 + o] = zs[o + o / R];
    __syncthreads();
  }
}

template <int R>
__global__ void __launch_bounds__(kStatelessP) k_dpd_bwd(StatelessArgs a) {
  extern __shared__ float4 smem_raw[];
  __shared__ float2 red[32];
  const uint64_t T = (uint64_t)R * blockDim.x;
  const uint64_t nt = (a.n + T - 1) / T;
  const size_t W = T + a.MT;
  float2* xs = reinterpret_cast<float2*>(smem_raw);
  float2* zs = xs + W;
  float2* gs = zs + (W + W / R + 2);
  for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    switch (a.MT) {
#define BWD_CASE(MTV) case MTV: bwd_tile<R, MTV>(a, t, xs, zs, gs, red); break;
      DPD_MT_CASES(BWD_CASE)
#undef BWD_CASE
      default: break;
    }
  }
}

// grad_h[k][m] = sum over tiles of partial[tile][k][m], in a fixed order.
// One CTA per tap (k, m): thread j sums the tile partials j, j + 256, .. in
// ascending order, then the 256 sums are combined by a tree of fixed shape
// (warp shuffles, then the 8 warp sums in order), so the result is the same
// on every run.
constexpr int kGhThreads = 256;
__global__ void __launch_bounds__(kGhThreads) k_gh_final(const float2* partial, uint64_t n_tiles, int K, int M,
                                                         int MT, float2* gh) {
  const int e = blockIdx.x;
  const int k = e / M, m = e % M;
  float2 s = make_float2(0.f, 0.f);
  for (uint64_t t = threadIdx.x; t < n_tiles; t += kGhThreads) {
    const float2 v = partial[(t * K + k) * MT + m];
    s.x += v.x;
    s.y += v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
  }
  __shared__ float2 ws[kGhThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = ws[0];
    for (int w = 1; w < kGhThreads / 32; ++w) {
      t.x += ws[w].x;
      t.y += ws[w].y;
    }
    gh[e] = t;
  }
}

// Resident CTAs of the stateless kernels: 16 per SM of the current device.
static uint64_t stateless_grid_cap() {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
    n_sm = 1;
  return 16ull * (uint64_t)n_sm;
}

static uint64_t stateless_tiles(uint64_t n) {
  const uint64_t T = (uint64_t)kStatelessR * kStatelessP;
  return (n + T - 1) / T;
}

size_t dpd_backward_scratch_elems(uint64_t n, int K, int M) {
  return stateless_tiles(n) * (size_t)K * dpd_supported_mt(M);
}

static cudaError_t stateless_common(StatelessArgs& a, const float2* h, int K, int M,
                                    const int* orders) {
  a.K = K;
  a.M = M;
  a.MT = dpd_supported_mt(M);
  if (!a.MT || K < 1 || K > kMaxBranches) return cudaErrorInvalidValue;
  for (int k = 0; k < K; ++k) a.orders[k] = orders[k];
  a.h = h;
  return cudaSuccess;
}

cudaError_t dpd_forward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M,
                                  const int* orders, float2* y, cudaStream_t s) {
  StatelessArgs a{};
  a.x = x;
  a.y = y;
  a.n = n;
  cudaError_t e = stateless_common(a, h, K, M, orders);
  if (e != cudaSuccess || n == 0) return e;
  const uint64_t T = (uint64_t)kStatelessR * kStatelessP;
  const size_t W = T + a.MT;
  const size_t smem = (W + W + W / kStatelessR + 2) * sizeof(float2);
  e = cudaFuncSetAttribute(k_dpd_fwd<kStatelessR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t nt = stateless_tiles(n);
  const unsigned grid = (unsigned)std::min<uint64_t>(nt, stateless_grid_cap());
  k_dpd_fwd<kStatelessR><<<grid, kStatelessP, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t dpd_backward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M,
                                   const int* orders, const float2* gy, float2* gx, float2* gh,
                                   float2* scratch, size_t scratch_elems, cudaStream_t s) {
  StatelessArgs a{};
  a.x = x;
  a.gy = gy;
  a.y = gx;
  a.gh = gh;
  a.n = n;
  cudaError_t e = stateless_common(a, h, K, M, orders);
  if (e != cudaSuccess) return e;
  if (scratch_elems < dpd_backward_scratch_elems(n, K, M)) return cudaErrorInvalidValue;
  a.partial = scratch;
  const uint64_t nt = stateless_tiles(n);
  if (n > 0) {
    const uint64_t T = (uint64_t)kStatelessR * kStatelessP;
    const size_t W = T + a.MT;
    const size_t smem = (W + 2 * (W + W / kStatelessR + 2)) * sizeof(float2);
    e = cudaFuncSetAttribute(k_dpd_bwd<kStatelessR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<uint64_t>(nt, stateless_grid_cap());
    k_dpd_bwd<kStatelessR><<<grid, kStatelessP, smem, s>>>(a);
  }
  k_gh_final<<<K * M, kGhThreads, 0, s>>>(a.partial, nt, K, M, a.MT, gh);
  return cudaGetLastError();
}

}  // namespace dfg
