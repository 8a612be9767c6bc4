// Shared host/device definitions of the dataflow engine.
//
// Every channel is a ring of `cap` slots of `tok` bytes in device memory.
// Its two counters live in device memory: wr = tokens ever written (initial
// tokens included), rd = tokens ever read; token i sits in slot i mod cap.
// Counters are 64-bit and only grow, so occupancy = wr - rd and
// free = cap - (wr - rd) are exact at any time.
//
// A channel in the paper's layout with a delay token (Sec. 3.2, Fig. 2) has
// one slot more: readers take token i from slot i mod cap (cap = 3r), writers
// put it in slot 1 + (i - 1) mod cap, so a write window never wraps, and the
// token that lands in slot cap is copied to slot 0 after its writer's body
// (the spill).  Writers see the channel through a descriptor whose ring starts
// at slot 1 and whose token index is shifted by wshift = 1; with that view
// every writer's ring arithmetic stays (i - wshift) mod cap.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/dfgpu.h"

namespace dfg {

constexpr int kMaxPorts = 16;

struct ChanDesc {          // immutable after finalize
  uint8_t* ring;
  uint64_t cap;            // slots
  uint64_t tok;            // bytes per token
  uint32_t rate;
  uint32_t id;             // index into the counter array
  uint32_t wshift;         // 1: writer view of a delay channel in the paper's layout
  uint32_t pad_;
};

struct EngineDev {          // device-resident engine state
  unsigned long long fired_total;
  int32_t status;           // DF_OK or the first device-side error
  int32_t status_where;     // which kernel / wait reported it
  // Arrivals at the persistent kernel's grid barriers, never reset while the
  // engine runs without an error (kBarrierError is added with every error).
  unsigned long long bar_arrive;
  unsigned int exit_count;      // persistent-kernel CTAs that have finished their last step
  unsigned int pad_;
  // Published counters for concurrent host I/O: a copy of the counter array
  // taken when a step has finished (all its bodies done).  Plans commit a
  // step's counters before its bodies move the data, so a push or pop that
  // runs beside the steps takes the other side's counter from here.
  uint64_t* ctr;
  uint64_t* pub;            // mapped host memory: the host reads it without a copy
  uint32_t n_words;         // 2 per channel
};

// where-codes for EngineDev::status_where
enum : int32_t { kWhereMdPipe = 1, kWhereGridBarrier = 2, kWhereDpd = 3, kWhereImgStage = 4 };

// Virtual grid: block index and block count of a phase (the launch's own grid
// for the per-phase kernels, the persistent kernel's grid otherwise).
struct Grid {
  uint32_t b, n;
};

__host__ __device__ inline uint64_t* wr_ptr(uint64_t* ctr, uint32_t ch) { return ctr + 2 * ch; }
__host__ __device__ inline uint64_t* rd_ptr(uint64_t* ctr, uint32_t ch) { return ctr + 2 * ch + 1; }

__host__ __device__ inline uint8_t* slot_ptr(const ChanDesc& c, uint64_t token_index) {
  return c.ring + ((token_index - c.wshift) % c.cap) * c.tok;
}

// Copy of slot cap into slot 0 after a write window reached slot cap (Fig. 2).
// The writer's plan keeps its counter from before the step (wr_before); the
// step wrote tokens wr_before .. wr-1, and the one among them whose index is
// a multiple of cap (at most one: a step writes at most cap tokens) sits in
// slot cap.
struct SpillArgs {
  uint8_t* ring;            // slot 0 of the buffer (reader view)
  uint64_t cap, tok;
  const uint64_t* wr_before;
  const uint64_t* ctr;
  uint32_t id;
  uint32_t unit;            // copy granularity in bytes: 16, 4 or 1
};

#ifdef __CUDACC__
// Added to bar_arrive with every recorded error: CTAs waiting at a grid
// barrier see it in the word they poll and leave.
constexpr unsigned long long kBarrierError = 1ull << 62;

__device__ inline void set_status(EngineDev* e, int32_t code, int32_t where) {
  if (atomicCAS(&e->status, 0, code) == 0) e->status_where = where;
  __threadfence();
  atomicAdd(&e->bar_arrive, kBarrierError);
}
#endif

// ------------------------------------------------------------------ copy ----
struct CopyPlan { uint64_t n; uint64_t rd0; uint64_t wr0[kMaxPorts]; };

struct CopyArgs {
  ChanDesc in;
  ChanDesc out[kMaxPorts];
  int n_out;
  int unit;                 // copy granularity in bytes: 16, 4 or 1
  uint64_t* ctr;
  EngineDev* eng;
  CopyPlan* plan;
};

// ---------------------------------------------------------- image actors ----
// The paper's motion pipeline (Sec. 4.1) as three static actors on u8 frames.
struct ImgPlan {
  uint64_t n;
  uint64_t rd0[2], wr0[kMaxPorts];          // token index of this step's first frame
  uint64_t slot_in[2], slot_out[kMaxPorts];  // its ring slot (index mod capacity)
};

struct ImgArgs {
  int kind;                 // DF_GAUSS5, DF_THRES, DF_MED5
  ChanDesc in[2];
  int n_in;
  ChanDesc out[kMaxPorts];
  int n_out;
  int W, H, thr;
  int dedup;                // Thres: in[1] is in[0]'s stream delayed by one token (same broadcast writer)
  int binary_in;            // Med: every input byte is 0 or 255 (written by Thres, initial tokens binary)
  long long wait_limit_ns;  // bound of every device-side wait
  uint64_t* ctr;
  EngineDev* eng;
  ImgPlan* plan;
};

// output rows per work item: 32, or 16 for frames wider than 1024 pixels (the
// shared memory of a CTA then stays under 227 KB up to the widest frame)
__host__ __device__ constexpr int img_band(int W) { return W <= 1024 ? 32 : 16; }
constexpr int kImgThreads = 256;
constexpr int kImgMaxWidth = 2048;
// staging buffers of an image body CTA: the band being computed and the
// next kImgBufs - 1 being loaded
constexpr int kImgBufs = 2;
// shared memory of an image body CTA: kImgBufs staging buffers of input rows
// (band + 2-row halo each side)
__host__ __device__ constexpr size_t img_smem_bytes(int W) {
  return kImgBufs * (size_t)(img_band(W) + 4) * W + 16;
}

// --------------------------------------------------- fused predistorter ----
constexpr int kMaxBranches = DF_MAX_BRANCHES;
constexpr int kMaxTaps = DF_MAX_TAPS;

struct DpdPlanHdr {
  uint64_t n;               // firings this step
  uint64_t rd_data0;        // data token index of firing 0
  uint64_t wr_out0;         // output token index of firing 0
  uint64_t slot_data0;      // rd_data0 mod data capacity
  uint64_t slot_out0;       // wr_out0 mod output capacity
  uint32_t parity_in;       // history buffer the body reads
  uint32_t pad;
  int32_t last[kMaxBranches];  // latest firing of the step with branch k active, -1: none
};

struct DpdArgs {            // one per predistorter actor, stored in device memory
  ChanDesc ctrl, data, out;  // ctrl.ring == nullptr: static actor, every firing has mask 1
  uint64_t* ctr;
  EngineDev* eng;
  int K, M, MT;             // MT = padded tap count of the kernel instantiation
  uint32_t L;               // samples per block
  uint32_t n_max;           // capacity of the per-firing arrays
  int orders[kMaxBranches];
  const float4* h;          // K * MT taps {hx, hx, hy, hy} (zero padded beyond M)
  DpdPlanHdr* plan;
  uint32_t* masks;          // [n_max]
  uint32_t* rank;           // [K][n_max]: active firings of branch k before firing i
  uint32_t* act;            // [K][n_max]: firing index of the a-th active block of k
  int32_t* prev;            // [K][n_max]: latest earlier firing of the step with k active, -1: none
  uint32_t* cnt;            // [K]: active firings of k this step
  float2* hist;             // [2][K][MT-1]: raw input samples preceding the batch
  uint32_t* parity;         // which half of hist is current
};

// --------------------------------------- bitmask-controlled dynamic actors ----
// Poly (in 0 control, in 1 data -> out k = branch k) and Adder (in 0 control,
// in k+1 = branch k -> out 0) of the expanded predistorter network.  Regular
// port p is active in a firing iff bit[p] of its control token is set (bit -1:
// always); an active port moves `rate` tokens.
constexpr int kDynPorts = kMaxBranches + 1;

struct DynPlanHdr {
  uint64_t n;                     // firings this step
  uint64_t base[kDynPorts];       // rd (inputs) / wr (outputs) of each port before the step
};

struct DynArgs {
  ChanDesc ctrl;
  ChanDesc port[kDynPorts];
  int is_out[kDynPorts];
  int bit[kDynPorts];
  int np;                         // regular ports
  int kind;                       // DF_DPD_POLY or DF_DPD_ADD
  int K;
  int orders[kMaxBranches];
  uint32_t L;                     // samples per token
  uint32_t n_max;
  uint64_t* ctr;
  EngineDev* eng;
  DynPlanHdr* plan;
  uint32_t* masks;                // [n_max]
  uint32_t* rank;                 // [np][n_max] active firings of port p before firing i
};

// ----------------------------------------------------- motion detector ----
struct MdPlanHdr {
  uint64_t n_cand;          // frames the main kernel processes this step
  uint64_t rd_cur0, rd_prev0, wr_rec0, wr_cnt0;
  uint64_t free_rec;        // free record slots at plan time
};

struct MdArgs {
  ChanDesc cur, prev, rec, cnt;
  uint64_t* ctr;
  EngineDev* eng;
  int W, H, thr;
  int words;                // W / 32
  int tiles_x, tiles_y, n_tiles;
  int strips;               // ceil(H / 16)
  int dedup;                // prev channel == cur channel delayed by one token
  int shared_rows;          // dedup and the current ring is under 2 GiB: 8-frame units
  uint32_t n_max;
  MdPlanHdr* plan;
  uint16_t* counts;         // [n_max][n_tiles]
  uint32_t* frame_tot;      // [n_max] records per frame
  uint64_t* frame_off;      // [n_max + 1] exclusive scan of frame_tot
  long long wait_limit_ns;  // bound of every device-side wait
};

// ------------------------------------------------ persistent step kernel ----
constexpr int kPersistThreads = 256;
enum : int { kPersistCopy = 1, kPersistDpd = 2, kPersistDyn = 3, kPersistMd = 4, kPersistImg = 5,
             kPersistSpill = 6 };

struct PersistOp {            // one entry of the device-side step program
  int kind;
  int n;                      // predistorter group size
  const void* args;           // CopyArgs / DpdArgs[n] / DynArgs / MdArgs / ImgArgs / SpillArgs[n]
  const uint16_t* order;      // predistorter group: the body's actor order
};

// --------------------------------------- programmatic dependent launch ----
// A kernel launched with programmatic stream serialisation may start while
// the previous kernel of the stream is still running; it must wait for that
// kernel's completion and memory (griddep_wait) before it touches any data an
// earlier kernel writes.  griddep_launch lets the next such kernel start.
// Both are no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// ----------------------------------------------------------- launchers ----
cudaError_t launch_set_u64(uint64_t* p, uint64_t v, cudaStream_t s);
cudaError_t launch_add_u64(uint64_t* p, uint64_t v, cudaStream_t s);
cudaError_t launch_publish(EngineDev* e, cudaStream_t s);   // pub = ctr after a step
cudaError_t launch_spill(const SpillArgs& a, cudaStream_t s);
cudaError_t launch_copy(const CopyArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                        cudaEvent_t ev1 = nullptr);

cudaError_t launch_dpd_plan(const DpdArgs* args_dev, int n_actors, cudaStream_t s, bool pdl = false);
cudaError_t launch_dpd_body(const DpdArgs* args_dev, const uint16_t* order, int n_actors, uint32_t tile,
                            uint32_t threads, int max_mt, int n_sm, cudaStream_t s, bool pdl = false);
int dpd_supported_mt(int M);   // padded tap count used for M (0 = unsupported)
cudaError_t dpd_prepare();     // one-time kernel attributes (outside graph capture)

cudaError_t launch_dyn(const DynArgs& a, int n_sm, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                       cudaEvent_t ev1 = nullptr);
struct MdTmaGeom {
  int pitch;                 // staged bytes per row: panel pixels + 2 halo tile columns
};
struct MdTma {               // tensor maps of the frame rings for the TMA main kernel
  CUtensorMap unit;          // current ring, all frames of a work unit per box
  CUtensorMap cur, prev;     // one frame per box
  MdTmaGeom geo;
  size_t smem;               // dynamic shared memory of a CTA
  int blocks_per_sm;
  int ok;                    // 0: the register-staged main kernel runs instead
};
cudaError_t launch_md_step(const MdArgs& a, const MdTma* tma, int n_sm, cudaStream_t s,
                           cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
cudaError_t md_prepare(int W);     // one-time kernel attributes (outside graph capture)
cudaError_t launch_img(const ImgArgs& a, int n_sm, cudaStream_t s);
cudaError_t img_prepare();         // one-time kernel attributes (outside graph capture)
cudaError_t md_tma_prepare(const MdArgs& a, MdTma* t);   // tensor maps + attributes
cudaError_t launch_md_main_tma(const MdArgs& a, const MdTma& t, int n_sm, cudaStream_t s, bool pdl);
size_t md_smem_bytes(int W);

cudaError_t persistent_prepare(size_t smem);
size_t persistent_smem(int mtmax, int max_group);
cudaError_t launch_persistent(const PersistOp* ops, int n_ops, EngineDev* eng, int64_t n_steps,
                              long long limit_ns, int mtmax, size_t smem, int n_sm, int per_sm_cap,
                              bool publish, cudaStream_t s);
cudaError_t launch_barrier_selftest(EngineDev* eng, long long limit_ns, cudaStream_t s);

cudaError_t dpd_forward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M,
                                  const int* orders, float2* y, cudaStream_t s);
cudaError_t dpd_backward_stateless(const float2* x, uint64_t n, const float2* h, int K, int M,
                                   const int* orders, const float2* gy, float2* gx, float2* gh,
                                   float2* scratch, size_t scratch_elems, cudaStream_t s);
size_t dpd_backward_scratch_elems(uint64_t n, int K, int M);
size_t dpd_mse_partial_elems(uint64_t n);
cudaError_t dpd_mse_forward(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                            const float2* target, float2* resid, float* loss, float* partial, cudaStream_t s);
cudaError_t dpd_mse_forward_f64(const double2* x, uint64_t n, const double2* h, int K, int M, const int* orders,
                                const double2* target, double2* resid, double* loss, double* partial,
                                cudaStream_t s);
cudaError_t dpd_mse_backward(const float2* x, uint64_t n, const float2* h, int K, int M, const int* orders,
                             const float2* resid, const float* grad_loss, float2* gh, float2* scratch,
                             size_t scratch_elems, cudaStream_t s);
cudaError_t dpd_mse_backward_f64(const double2* x, uint64_t n, const double2* h, int K, int M, const int* orders,
                                 const double2* resid, const double* grad_loss, double2* gh, double2* scratch,
                                 size_t scratch_elems, cudaStream_t s);
cudaError_t dpd_forward_stateless_f64(const double2* x, uint64_t n, const double2* h, int K, int M,
                                      const int* orders, double2* y, cudaStream_t s);
cudaError_t dpd_backward_stateless_f64(const double2* x, uint64_t n, const double2* h, int K, int M,
                                       const int* orders, const double2* gy, double2* gx, double2* gh,
                                       double2* scratch, size_t scratch_elems, cudaStream_t s);

}  // namespace dfg
