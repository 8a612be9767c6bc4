// Stateless differentiable predistorter (the Sec. 4.2 network with every
// branch active, on one signal, zero history) and its adjoint, in float32
// (complex64) or float64 (complex128) arithmetic.  The float64 form exists so
// that the adjoint can be checked by finite differences at full precision.
//
// Forward, per tile of T = R * blockDim.x outputs: the x window with MT-1
// samples of history is staged in shared memory; per branch the branch signal
// z = |x|^(o-1) x is formed in a padded shared buffer, and each thread
// accumulates R consecutive outputs of the M-tap complex FIR.
// Adjoint, per tile: with g = dL/dy (PyTorch's complex convention), the tap
// gradient partial sum_n g[n] conj(z_k[n-m]) of the tile is reduced over the
// CTA into partial[tile][k][m]; gz_k[j] = sum_m conj(h[k,m]) g[j+m] gives
// grad_x by the chain rule through z = u^q x (u = |x|^2).  A second kernel
// sums the tile partials of each tap in a fixed order.
// Fused loss of the fit (L = mean |P_h(x) - t|^2): the forward writes the
// residual d = y - t instead of y and each tile's sum of |d|^2, a second
// kernel sums the tiles in a fixed order; the adjoint then takes
// dL/dy = d * (2 g / n) with the upstream scalar g read from device memory.
#include <algorithm>
#include "dpd_dev.cuh"

namespace dfg {
namespace {

template <class V> struct Cx;
template <> struct Cx<float2> {
  using S = float;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
};
template <> struct Cx<double2> {
  using S = double;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }
};

template <class V> __device__ __forceinline__ V czero() { return Cx<V>::make(0, 0); }

// acc += h * z
template <class V> __device__ __forceinline__ V cmac(V acc, V h, V z) {
  using C = Cx<V>;
  acc.x = C::fm(h.x, z.x, acc.x);
  acc.x = C::fm(-h.y, z.y, acc.x);
  acc.y = C::fm(h.x, z.y, acc.y);
  acc.y = C::fm(h.y, z.x, acc.y);
  return acc;
}
// acc += a * conj(b)
template <class V> __device__ __forceinline__ V cmac_conj_b(V acc, V a, V b) {
  using C = Cx<V>;
  acc.x = C::fm(a.x, b.x, acc.x);
  acc.x = C::fm(a.y, b.y, acc.x);
  acc.y = C::fm(a.y, b.x, acc.y);
  acc.y = C::fm(-a.x, b.y, acc.y);
  return acc;
}

// |x|^(2q) x with u = |x|^2 raised by repeated products
template <class V> __device__ __forceinline__ V psi_q(V x, int q) {
  using S = typename Cx<V>::S;
  const S u = Cx<V>::fm(x.x, x.x, x.y * x.y);
  S p = 1;
  for (int i = 0; i < q; ++i) p *= u;
  return Cx<V>::make(p * x.x, p * x.y);
}

// Shared windows are padded with one element after every R elements so that
// threads reading at stride R elements hit distinct banks.
// Causal chunk: acc[r] += sum_{m<MC} h[m] * zs[v], v = p*R + shift + r - m + MC - 1;
// taps m >= m_valid are zero.
template <class V, int R, int MC>
__device__ __forceinline__ void fir_causal(V (&acc)[R], const V* __restrict__ zs, int p, int shift,
                                           const V* __restrict__ h, int m_valid) {
  V hk[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) hk[m] = m < m_valid ? h[m] : czero<V>();
  const V* zb = zs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const V z = zb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) acc[r] = cmac(acc[r], hk[m], z);
    }
  }
}

// Anti-causal chunk with conjugated taps: acc[r] += sum_m conj(h[m]) * gs[v], v = p*R + shift + r + m.
template <class V, int R, int MC>
__device__ __forceinline__ void fir_anticausal_conj(V (&acc)[R], const V* __restrict__ gs, int p, int shift,
                                                    const V* __restrict__ h, int m_valid) {
  V ck[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const V t = m < m_valid ? h[m] : czero<V>();
    ck[m] = Cx<V>::make(t.x, -t.y);
  }
  const V* gb = gs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const V g = gb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = s - r;
      if (m >= 0 && m < MC) acc[r] = cmac(acc[r], ck[m], g);
    }
  }
}

// Tap-gradient chunk: ph[m] += sum_r g[r] * conj(zs[v]), v = p*R + shift + r - m + MC - 1.
template <class V, int R, int MC>
__device__ __forceinline__ void gh_chunk(V (&ph)[MC], const V (&gr)[R], const V* __restrict__ zs, int p,
                                         int shift) {
  const V* zb = zs + p * (R + 1) + shift + shift / R;
#pragma unroll
  for (int s = 0; s < R + MC - 1; ++s) {
    const V z = zb[s + s / R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = r + MC - 1 - s;
      if (m >= 0 && m < MC) ph[m] = cmac_conj_b(ph[m], gr[r], z);
    }
  }
}

// FIR of one branch over a staged window, MT <= 16 in one chunk, MT == 32 in two.
template <class V, int R, int MT>
__device__ __forceinline__ void fir_branch(V (&acc)[R], const V* zs, int p, const V* h, int M) {
  if constexpr (MT <= 16) {
    fir_causal<V, R, MT>(acc, zs, p, 0, h, M);
  } else {
    fir_causal<V, R, 16>(acc, zs, p, 16, h, M);
    fir_causal<V, R, 16>(acc, zs, p, 0, h + 16, M - 16);
  }
}

constexpr int kStatelessR = 8;
constexpr int kStatelessP = 128;

template <class V>
struct StatelessArgs {
  using S = typename Cx<V>::S;
  const V* x;
  const V* gy;
  V* y;                 // forward output (the residual with target) or grad_x
  V* partial;           // [tiles][K][MT] tap-gradient partial sums
  V* gh;                // [K][M]
  const V* h;           // [K][M] taps (unpadded: tap m >= M contributes zero)
  const V* target;      // forward: y - target is written, with per-tile sums of its |.|^2
  S* loss_partial;      // [tiles]
  const S* gscale;      // adjoint: gy is scaled by gmult * gscale[0] when set
  S gmult;
  uint64_t n;
  int K, M, MT;
  int orders[kMaxBranches];
};

// Deterministic block sum of one value per thread (thread 0 gets the result).
template <class V> __device__ V block_sum(V v, V* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if (lane == 0) red[wid] = v;
  __syncthreads();
  V s = czero<V>();
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) {
      s.x += red[w].x;
      s.y += red[w].y;
    }
  __syncthreads();
  return s;
}

template <class V, int R, int MT>
__device__ void fwd_tile(const StatelessArgs<V>& a, uint64_t tile, V* xs, V* zs) {
  const int P = blockDim.x, p = threadIdx.x;
  const uint64_t T = (uint64_t)R * P;
  const uint64_t t0 = tile * T;
  const int len = (int)min(T, a.n - t0);
  const int W = (int)T + MT - 1;
  for (int v = p; v < W; v += P) {
    const int64_t pos = (int64_t)t0 - (MT - 1) + v;
    xs[v] = (pos >= 0 && pos < (int64_t)(t0 + len)) ? a.x[pos] : czero<V>();
  }
  __syncthreads();
  V acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = czero<V>();
  for (int k = 0; k < a.K; ++k) {
    const int q = (a.orders[k] - 1) >> 1;
    for (int v = p; v < W; v += P) zs[v + v / R] = psi_q(xs[v], q);
    __syncthreads();
    fir_branch<V, R, MT>(acc, zs, p, a.h + (size_t)k * a.M, a.M);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) zs[p * (R + 1) + r] = acc[r];
  __syncthreads();
  if (!a.target) {
    for (int o = p; o < len; o += P) a.y[t0 + o] = zs[o + o / R];
  } else {
    using S = typename Cx<V>::S;
    S e2 = 0;
    for (int o = p; o < len; o += P) {
      const V y = zs[o + o / R], t = a.target[t0 + o];
      const V d = Cx<V>::make(y.x - t.x, y.y - t.y);
      a.y[t0 + o] = d;
      e2 = Cx<V>::fm(d.x, d.x, Cx<V>::fm(d.y, d.y, e2));
    }
    __shared__ V red[32];
    const V sum = block_sum(Cx<V>::make(e2, 0), red);
    if (threadIdx.x == 0) a.loss_partial[tile] = sum.x;
  }
  __syncthreads();
}

template <class V, int R>
__global__ void __launch_bounds__(kStatelessP) k_dpd_fwd(StatelessArgs<V> a) {
  extern __shared__ float4 smem_raw[];
  const uint64_t T = (uint64_t)R * blockDim.x;
  const uint64_t nt = (a.n + T - 1) / T;
  V* xs = reinterpret_cast<V*>(smem_raw);
  V* zs = xs + (T + a.MT);
  for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    switch (a.MT) {
#define FWD_CASE(MTV) case MTV: fwd_tile<V, R, MTV>(a, t, xs, zs); break;
      DPD_MT_CASES(FWD_CASE)
#undef FWD_CASE
      default: break;
    }
  }
}

template <class V, int R, int MC>
__device__ void gh_reduce_chunk(const StatelessArgs<V>& a, uint64_t tile, int k, int m0, const V (&gr)[R],
                                const V* zs, int shift, V* red) {
  V ph[MC];
#pragma unroll
  for (int m = 0; m < MC; ++m) ph[m] = czero<V>();
  gh_chunk<V, R, MC>(ph, gr, zs, threadIdx.x, shift);
#pragma unroll
  for (int m = 0; m < MC; ++m) {
    const V s = block_sum(ph[m], red);
    if (threadIdx.x == 0) a.partial[(tile * a.K + k) * a.MT + m0 + m] = s;
  }
}

template <class V, int R, int MT>
__device__ void bwd_tile(const StatelessArgs<V>& a, uint64_t tile, V* xs, V* zs, V* gs, V* red) {
  using S = typename Cx<V>::S;
  using C = Cx<V>;
  const int P = blockDim.x, p = threadIdx.x;
  const uint64_t T = (uint64_t)R * P;
  const uint64_t t0 = tile * T;
  const int len = (int)min(T, a.n - t0);
  const int W = (int)T + MT - 1;
  const S gsc = a.gscale ? a.gmult * a.gscale[0] : S(1);
  for (int v = p; v < W; v += P) {
    const int64_t pos = (int64_t)t0 - (MT - 1) + v;
    xs[v] = (pos >= 0 && pos < (int64_t)(t0 + len)) ? a.x[pos] : czero<V>();
    const uint64_t gp = t0 + v;       // g window [t0, t0 + T + MT - 1), zero beyond n
    V gv = gp < a.n ? a.gy[gp] : czero<V>();
    gv.x *= gsc;
    gv.y *= gsc;
    gs[v + v / R] = gv;
  }
  __syncthreads();
  V gr[R], gx[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    gr[r] = (p * R + r < len) ? gs[p * (R + 1) + r] : czero<V>();
    gx[r] = czero<V>();
  }
  for (int k = 0; k < a.K; ++k) {
    const int q = (a.orders[k] - 1) >> 1;
    for (int v = p; v < W; v += P) zs[v + v / R] = psi_q(xs[v], q);
    __syncthreads();
    const V* hk = a.h + (size_t)k * a.M;
    V gz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) gz[r] = czero<V>();
    if constexpr (MT <= 16) {
      gh_reduce_chunk<V, R, MT>(a, tile, k, 0, gr, zs, 0, red);
      fir_anticausal_conj<V, R, MT>(gz, gs, p, 0, hk, a.M);
    } else {
      gh_reduce_chunk<V, R, 16>(a, tile, k, 0, gr, zs, 16, red);
      gh_reduce_chunk<V, R, 16>(a, tile, k, 16, gr, zs, 0, red);
      fir_anticausal_conj<V, R, 16>(gz, gs, p, 0, hk, a.M);
      fir_anticausal_conj<V, R, 16>(gz, gs, p, 16, hk + 16, a.M - 16);
    }
    if (a.y) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const V x = xs[p * R + r + MT - 1];
        const S u = C::fm(x.x, x.x, x.y * x.y);
        S uq1 = 1;
        for (int i = 0; i + 1 < q; ++i) uq1 *= u;
        const S uq = q > 0 ? uq1 * u : S(1);
        const S c1 = (q + 1) * uq;
        gx[r].x = C::fm(c1, gz[r].x, gx[r].x);
        gx[r].y = C::fm(c1, gz[r].y, gx[r].y);
        if (q > 0) {
          const S c2 = q * uq1;
          const V x2 = C::make(x.x * x.x - x.y * x.y, 2 * x.x * x.y);
          // c2 * x^2 * conj(gz)
          gx[r].x = C::fm(c2, x2.x * gz[r].x + x2.y * gz[r].y, gx[r].x);
          gx[r].y = C::fm(c2, x2.y * gz[r].x - x2.x * gz[r].y, gx[r].y);
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

template <class V, int R>
__global__ void __launch_bounds__(kStatelessP) k_dpd_bwd(StatelessArgs<V> a) {
  extern __shared__ float4 smem_raw[];
  __shared__ V red[32];
  const uint64_t T = (uint64_t)R * blockDim.x;
  const uint64_t nt = (a.n + T - 1) / T;
  const size_t W = T + a.MT;
  V* xs = reinterpret_cast<V*>(smem_raw);
  V* zs = xs + W;
  V* gs = zs + (W + W / R + 2);
  for (uint64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    switch (a.MT) {
#define BWD_CASE(MTV) case MTV: bwd_tile<V, R, MTV>(a, t, xs, zs, gs, red); break;
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
template <class V>
__global__ void __launch_bounds__(kGhThreads) k_gh_final(const V* partial, uint64_t n_tiles, int K, int M, int MT,
                                                         V* gh) {
  const int e = blockIdx.x;
  const int k = e / M, m = e % M;
  V s = czero<V>();
  for (uint64_t t = threadIdx.x; t < n_tiles; t += kGhThreads) {
    const V v = partial[(t * K + k) * MT + m];
    s.x += v.x;
    s.y += v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
  }
  __shared__ V ws[kGhThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    V t = ws[0];
    for (int w = 1; w < kGhThreads / 32; ++w) {
      t.x += ws[w].x;
      t.y += ws[w].y;
    }
    gh[e] = t;
  }
}

// loss = (sum of the tile sums in a fixed order) / n: thread j sums tiles j,
// j + 256, .. in ascending order, then the 256 sums by a tree of fixed shape.
template <class S>
__global__ void __launch_bounds__(kGhThreads) k_loss_final(const S* partial, uint64_t n_tiles, uint64_t n,
                                                           S* loss) {
  S v = 0;
  for (uint64_t t = threadIdx.x; t < n_tiles; t += kGhThreads) v += partial[t];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __shared__ S ws[kGhThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    S t = ws[0];
    for (int w = 1; w < kGhThreads / 32; ++w) t += ws[w];
    *loss = n ? t / (S)n : S(0);
  }
}

// Resident CTAs of the stateless kernels: 16 per SM of the current device.
uint64_t stateless_grid_cap() {
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1)
    n_sm = 1;
  return 16ull * (uint64_t)n_sm;
}

uint64_t stateless_tiles(uint64_t n) {
  const uint64_t T = (uint64_t)kStatelessR * kStatelessP;
  return (n + T - 1) / T;
}

template <class V>
cudaError_t stateless_common(StatelessArgs<V>& a, const V* h, int K, int M, const int* orders) {
  a.K = K;
  a.M = M;
  a.MT = dpd_supported_mt(M);
  if (!a.MT || K < 1 || K > kMaxBranches) return cudaErrorInvalidValue;
  for (int k = 0; k < K; ++k) a.orders[k] = orders[k];
  a.h = h;
  return cudaSuccess;
}

template <class V>
cudaError_t forward_impl(const V* x, uint64_t n, const V* h, int K, int M, const int* orders, V* y,
                         cudaStream_t s, const V* target = nullptr, typename Cx<V>::S* loss = nullptr,
                         typename Cx<V>::S* loss_partial = nullptr) {
  StatelessArgs<V> a{};
  a.x = x;
  a.y = y;
  a.n = n;
  a.target = target;
  a.loss_partial = loss_partial;
  cudaError_t e = stateless_common(a, h, K, M, orders);
  if (e != cudaSuccess) return e;
  if (n == 0) {
    if (target) k_loss_final<typename Cx<V>::S><<<1, kGhThreads, 0, s>>>(loss_partial, 0, 0, loss);
    return cudaGetLastError();
  }
  const uint64_t T = (uint64_t)kStatelessR * kStatelessP;
  const size_t W = T + a.MT;
  const size_t smem = (W + W + W / kStatelessR + 2) * sizeof(V);
  e = cudaFuncSetAttribute(k_dpd_fwd<V, kStatelessR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<uint64_t>(stateless_tiles(n), stateless_grid_cap());
  k_dpd_fwd<V, kStatelessR><<<grid, kStatelessP, smem, s>>>(a);
  if (target) k_loss_final<typename Cx<V>::S><<<1, kGhThreads, 0, s>>>(loss_partial, stateless_tiles(n), n, loss);
  return cudaGetLastError();
}

template <class V>
cudaError_t backward_impl(const V* x, uint64_t n, const V* h, int K, int M, const int* orders, const V* gy, V* gx,
                          V* gh, V* scratch, size_t scratch_elems, cudaStream_t s,
                          const typename Cx<V>::S* gscale = nullptr, typename Cx<V>::S gmult = 1) {
  StatelessArgs<V> a{};
  a.x = x;
  a.gy = gy;
  a.gscale = gscale;
  a.gmult = gmult;
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
    const size_t smem = (W + 2 * (W + W / kStatelessR + 2)) * sizeof(V);
    e = cudaFuncSetAttribute(k_dpd_bwd<V, kStatelessR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<uint64_t>(nt, stateless_grid_cap());
    k_dpd_bwd<V, kStatelessR><<<grid, kStatelessP, smem, s>>>(a);
  }
  k_gh_final<V><<<K * M, kGhThreads, 0, s>>>(a.partial, nt, K, M, a.MT, gh);
  return cudaGetLastError();
}

}  // namespace

size_t dpd_backward_scratch_elems(uint64_t n, int K, int M) {
  return stateless_tiles(n) * (size_t)K * dpd_supported_mt(M);
}

cudaError_t dpd_forward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                                  float2* y, cudaStream_t s) {
  return forward_impl<float2>(x, n, h, K, M, orders, y, s);
}

cudaError_t dpd_forward_stateless_f64(const double2* x, uint64_t n, const double2* h, int K, int M,
                                      const int* orders, double2* y, cudaStream_t s) {
  return forward_impl<double2>(x, n, h, K, M, orders, y, s);
}

cudaError_t dpd_backward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                                   const float2* gy, float2* gx, float2* gh, float2* scratch, size_t scratch_elems,
                                   cudaStream_t s) {
  return backward_impl<float2>(x, n, h, K, M, orders, gy, gx, gh, scratch, scratch_elems, s);
}

cudaError_t dpd_backward_stateless_f64(const double2* x, uint64_t n, const double2* h, int K, int M,
                                       const int* orders, const double2* gy, double2* gx, double2* gh,
                                       double2* scratch, size_t scratch_elems, cudaStream_t s) {
  return backward_impl<double2>(x, n, h, K, M, orders, gy, gx, gh, scratch, scratch_elems, s);
}

size_t dpd_mse_partial_elems(uint64_t n) { return std::max<uint64_t>(1, stateless_tiles(n)); }

cudaError_t dpd_mse_forward(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                            const float2* target, float2* resid, float* loss, float* partial, cudaStream_t s) {
  return forward_impl<float2>(x, n, h, K, M, orders, resid, s, target, loss, partial);
}
cudaError_t dpd_mse_forward_f64(const double2* x, uint64_t n, const double2* h, int K, int M, const int* orders,
                                const double2* target, double2* resid, double* loss, double* partial,
                                cudaStream_t s) {
  return forward_impl<double2>(x, n, h, K, M, orders, resid, s, target, loss, partial);
}
cudaError_t dpd_mse_backward(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                             const float2* resid, const float* grad_loss, float2* gh, float2* scratch,
                             size_t scratch_elems, cudaStream_t s) {
  return backward_impl<float2>(x, n, h, K, M, orders, resid, nullptr, gh, scratch, scratch_elems, s, grad_loss,
                               n ? 2.0f / (float)n : 0.0f);
}
cudaError_t dpd_mse_backward_f64(const double2* x, uint64_t n, const double2* h, int K, int M, const int* orders,
                                 const double2* resid, const double* grad_loss, double2* gh, double2* scratch,
                                 size_t scratch_elems, cudaStream_t s) {
  return backward_impl<double2>(x, n, h, K, M, orders, resid, nullptr, gh, scratch, scratch_elems, s, grad_loss,
                                n ? 2.0 / (double)n : 0.0);
}

}  // namespace dfg
