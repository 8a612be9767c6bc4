// Host side of the engine: network construction and validation (Sec. 2.2,
// Sec. 3.2), planning of the device arena, the step program, and the host
// endpoints push / pop.
//
// Planning.  At finalize every channel ring, the counter array and the
// per-actor state are carved out of one device allocation, each piece aligned
// to 256 bytes.  The step program is a list of operations, one per actor in
// insertion order; consecutive fused-predistorter actors that share no
// channel form a group that is planned and fired by one plan launch and one
// body launch.  A step never returns to the host: rate decisions, scans,
// gathers and scatters are all device kernels reading the device counters.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace dfg;

namespace {

struct ActorH {
  int32_t kind = 0;
  std::vector<int32_t> in, out;       // channel per port, -1 = unconnected
  df_dpd_params dpd{};
  std::vector<float> h;               // K*M complex taps (host copy)
  df_md_params md{};
  df_img_params img{};
  uint32_t tile = 0, threads = 0;     // predistorter body configuration (0 = default)
};

struct ChanH {
  int32_t src, sport, dst, dport;
  uint32_t tok, rate, cap, init;
  bool eq1 = false;                   // the paper's layout (Eq. 1, Fig. 2)
  std::vector<uint8_t> init_data;
  ChanDesc desc{};                    // reader view
  ChanDesc wdesc{};                   // writer view (differs for a delay channel in the paper's layout)
  uint64_t slots() const { return (uint64_t)cap + (eq1 && init ? 1 : 0); }
};

enum OpKind { kOpCopy = 1, kOpDpd = 2, kOpMd = 3, kOpDyn = 4, kOpImg = 5 };

struct Op {
  OpKind kind;
  CopyArgs copy{};
  MdArgs md{};
  MdTma md_tma{};
  DynArgs dyn{};
  ImgArgs img{};
  DpdArgs* dpd_dev = nullptr;        // group args (device)
  int dpd_n = 0;                      // actors in the group
  int dpd_first_actor = -1;           // actor id of the first member
  const uint16_t* dpd_order = nullptr;  // the body's actor order (device; by padded tap count)
  int max_mt = 0;
  std::vector<SpillArgs> spills;      // Fig. 2 copies after the op's bodies
};

struct Piece {                        // one carve of the device arena
  size_t off = 0, bytes = 0;
};

}  // namespace

struct df_net {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool finalized = false;
  int n_sm = 148;
  std::vector<ActorH> actors;
  std::vector<ChanH> chans;
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  uint64_t* d_ctr = nullptr;
  uint64_t* d_pub = nullptr;          // counters published after each step (concurrent I/O),
  uint64_t* h_pub = nullptr;          // in mapped pinned host memory: d_pub is its device address
  // the counters only the host moves (wr of a source's channels, rd of a
  // sink's), kept by the pushing / popping thread after each of its calls
  std::vector<uint64_t> host_ctr;
  std::atomic<bool> io_used{false};   // a concurrent push or pop happened: publish every step
  EngineDev* d_eng = nullptr;
  std::vector<DpdArgs> dpd_host;      // one per predistorter actor (by dpd index)
  std::vector<int> dpd_index;         // actor id -> index in dpd_host (-1)
  DpdArgs* d_dpd = nullptr;           // device copy of dpd_host
  std::vector<Op> program;
  uint64_t* h_pin = nullptr;          // pinned staging (counters, status)
  uint64_t fired_seen = 0;            // fired_total as last read after all queued work
  bool fired_known = false;           // false after asynchronous runs and the autotuner
  // concurrent host I/O (DF_IO_CONCURRENT): [0] pushes, [1] pops, each on a
  // stream of its own, created on first use (counters are staged in pinned
  // memory of the calling thread, so several sources or sinks can be served
  // by threads of their own)
  cudaStream_t io_stream[2] = {nullptr, nullptr};
  std::mutex io_mu;
  std::map<std::pair<int64_t, uint32_t>, cudaGraphExec_t> graphs;
  long long wait_limit_ns = 1000000000LL;
  // kernel timing (df_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[4] = {0, 0, 0, 0};
  uint64_t prof_n[4] = {0, 0, 0, 0};
  // persistent step kernel: device-side program (built on first use)
  void* persist_mem = nullptr;
  PersistOp* d_persist_ops = nullptr;
  int persist_n_ops = 0, persist_mtmax = 16;
  int persist_per_sm = 0;             // CTAs per SM of the persistent grid (0: as many as fit)
  size_t persist_smem = 0;
};

namespace {


thread_local char g_last_error[256] = "";

df_status record_cuda(cudaError_t e, const char* what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  return DF_ECUDA;
}

#define DF_CUDA(x)                                       \
  do {                                                   \
    cudaError_t e_ = (x);                                \
    if (e_ != cudaSuccess) return record_cuda(e_, #x);   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_dynamic(int32_t kind) {
  return kind == DF_DPD || kind == DF_DPD_POLY || kind == DF_DPD_ADD;
}

int n_connected(const std::vector<int32_t>& v) {
  return (int)std::count_if(v.begin(), v.end(), [](int32_t c) { return c >= 0; });
}

bool dense(const std::vector<int32_t>& v) {
  for (int32_t c : v)
    if (c < 0) return false;
  return true;
}

uint32_t tiles_per_frame(const df_md_params& m) {
  return (uint32_t)(((m.height + 15) / 16) * ((m.width + 15) / 16));
}

df_status validate_actor(const df_net* net, int a) {
  const ActorH& A = net->actors[a];
  if (!dense(A.in) || !dense(A.out)) return DF_EINVAL;
  auto ch = [&](int32_t id) -> const ChanH& { return net->chans[id]; };
  switch (A.kind) {
    case DF_SOURCE:
      if (!A.in.empty() || A.out.empty()) return DF_EINVAL;
      return DF_OK;
    case DF_SINK:
      if (A.in.size() != 1 || !A.out.empty()) return DF_EINVAL;
      return DF_OK;
    case DF_GAUSS5:
    case DF_THRES:
    case DF_MED5: {
      const size_t n_in = A.kind == DF_THRES ? 2 : 1;
      if (A.in.size() != n_in || A.out.empty() || (int)A.out.size() > kMaxPorts) return DF_EINVAL;
      if (A.kind == DF_THRES && A.out.size() != 1) return DF_EINVAL;
      const uint64_t fb = (uint64_t)A.img.width * A.img.height;
      const uint32_t r = ch(A.in[0]).rate;
      for (int32_t c : A.in)
        if (ch(c).tok != fb || ch(c).rate != r) return DF_EINVAL;
      for (int32_t c : A.out)
        if (ch(c).tok != fb || ch(c).rate != r) return DF_EINVAL;
      return DF_OK;
    }
    case DF_COPY: {
      if (A.in.size() != 1 || A.out.empty() || (int)A.out.size() > kMaxPorts) return DF_EINVAL;
      const ChanH& i = ch(A.in[0]);
      for (int32_t o : A.out)
        if ((uint64_t)i.tok * i.rate != (uint64_t)ch(o).tok * ch(o).rate) return DF_EINVAL;
      return DF_OK;
    }
    case DF_DPD: {
      if (A.in.size() != 2 || A.out.size() != 1) return DF_EINVAL;
      const df_dpd_params& p = A.dpd;
      const uint64_t blk = (uint64_t)p.block_len * 8;
      const ChanH &c = ch(A.in[0]), &d = ch(A.in[1]), &o = ch(A.out[0]);
      if (c.tok != 4 || c.rate != 1) return DF_EINVAL;
      if (d.tok != blk || d.rate != 1 || o.tok != blk || o.rate != 1) return DF_EINVAL;
      return DF_OK;
    }
    case DF_MD: {
      if (A.in.size() != 2 || A.out.size() != 2) return DF_EINVAL;
      const df_md_params& m = A.md;
      const uint64_t fb = (uint64_t)m.width * m.height;
      const ChanH &c = ch(A.in[0]), &p = ch(A.in[1]), &r = ch(A.out[0]), &n = ch(A.out[1]);
      if (c.tok != fb || p.tok != fb || c.rate != 1 || p.rate != 1) return DF_EINVAL;
      if (r.tok != 8 || r.rate != tiles_per_frame(m)) return DF_EINVAL;
      if (n.tok != 4 || n.rate != 1) return DF_EINVAL;
      return DF_OK;
    }
    case DF_DPD_POLY: {
      const df_dpd_params& p = A.dpd;
      const uint64_t blk = (uint64_t)p.block_len * 8;
      if (A.in.size() != 2 || (int)A.out.size() != p.K) return DF_EINVAL;
      if (ch(A.in[0]).tok != 4 || ch(A.in[0]).rate != 1) return DF_EINVAL;
      if (ch(A.in[1]).tok != blk || ch(A.in[1]).rate != 1) return DF_EINVAL;
      for (int32_t o : A.out)
        if (ch(o).tok != blk || ch(o).rate != 1) return DF_EINVAL;
      return DF_OK;
    }
    case DF_DPD_ADD: {
      const df_dpd_params& p = A.dpd;
      const uint64_t blk = (uint64_t)p.block_len * 8;
      if ((int)A.in.size() != p.K + 1 || A.out.size() != 1) return DF_EINVAL;
      if (ch(A.in[0]).tok != 4 || ch(A.in[0]).rate != 1) return DF_EINVAL;
      for (size_t i = 1; i < A.in.size(); ++i)
        if (ch(A.in[i]).tok != blk || ch(A.in[i]).rate != 1) return DF_EINVAL;
      if (ch(A.out[0]).tok != blk || ch(A.out[0]).rate != 1) return DF_EINVAL;
      return DF_OK;
    }
    case DF_DPD_FIR: {
      const df_dpd_params& p = A.dpd;
      const uint64_t blk = (uint64_t)p.block_len * 8;
      if (A.in.size() != 1 || A.out.size() != 1) return DF_EINVAL;
      if (p.branch < 0 || p.branch >= p.K) return DF_EINVAL;
      if (ch(A.in[0]).tok != blk || ch(A.in[0]).rate != 1) return DF_EINVAL;
      if (ch(A.out[0]).tok != blk || ch(A.out[0]).rate != 1) return DF_EINVAL;
      return DF_OK;
    }
    default:
      return DF_EINVAL;
  }
}

// The engine word after all queued work, with one copy into the pinned
// staging and one wait: the firing total and the device status.
static_assert(offsetof(EngineDev, fired_total) == 0 && offsetof(EngineDev, status) == 8,
              "engine word layout");
df_status read_engine(df_net* net, uint64_t* total, int32_t* status) {
  DF_CUDA(cudaMemcpyAsync(net->h_pin, net->d_eng, 16, cudaMemcpyDeviceToHost, net->stream));
  DF_CUDA(cudaStreamSynchronize(net->stream));
  *total = net->h_pin[0];
  std::memcpy(status, reinterpret_cast<const uint8_t*>(net->h_pin) + 8, sizeof(int32_t));
  net->fired_seen = *total;
  net->fired_known = true;
  return DF_OK;
}

df_status fail_if_device_error(df_net* net) {
  uint64_t total;
  int32_t st;
  const df_status e = read_engine(net, &total, &st);
  return e != DF_OK ? e : st;
}

df_status read_counters(df_net* net, int32_t ch, uint64_t* wr, uint64_t* rd,
                        cudaStream_t s = nullptr, uint64_t* pin = nullptr) {
  if (!s) s = net->stream;
  if (!pin) pin = net->h_pin;
  DF_CUDA(cudaMemcpyAsync(pin, net->d_ctr + 2 * ch, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  DF_CUDA(cudaStreamSynchronize(s));
  *wr = pin[0];
  *rd = pin[1];
  return DF_OK;
}

// Copy `bytes` bytes between a linear buffer and a ring starting at token `t`.
df_status ring_copy(df_net* net, const ChanDesc& c, uint64_t t, void* lin, uint64_t n_tok,
                    bool to_ring, cudaStream_t s = nullptr) {
  if (!s) s = net->stream;
  const uint64_t slot = (t - c.wshift) % c.cap;
  const uint64_t first = std::min<uint64_t>(n_tok, c.cap - slot);
  uint8_t* ring0 = c.ring + slot * c.tok;
  uint8_t* l = static_cast<uint8_t*>(lin);
  if (first) {
    if (to_ring)
      DF_CUDA(cudaMemcpyAsync(ring0, l, first * c.tok, cudaMemcpyDefault, s));
    else
      DF_CUDA(cudaMemcpyAsync(l, ring0, first * c.tok, cudaMemcpyDefault, s));
  }
  if (n_tok > first) {
    const uint64_t rest = n_tok - first;
    if (to_ring)
      DF_CUDA(cudaMemcpyAsync(c.ring, l + first * c.tok, rest * c.tok, cudaMemcpyDefault, s));
    else
      DF_CUDA(cudaMemcpyAsync(l + first * c.tok, c.ring, rest * c.tok, cudaMemcpyDefault, s));
  }
  return DF_OK;
}

// Untuned tile: 16 outputs per lane for long blocks, 8 otherwise (the measured
// best on 2^20-sample blocks and on 1-256 Ki-sample blocks respectively).
uint32_t default_tile(const DpdArgs& a) { return a.L >= 16384 ? 4096 : 2048; }

cudaEvent_t take_event(df_net* net) {
  if (!net->ev_free.empty()) {
    cudaEvent_t e = net->ev_free.back();
    net->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Timing pair for `what` when profiling is on (both null otherwise).
std::pair<cudaEvent_t, cudaEvent_t> prof_pair(df_net* net, int what, bool capturing) {
  if (!net->prof || capturing) return {nullptr, nullptr};
  std::pair<cudaEvent_t, cudaEvent_t> p{take_event(net), take_event(net)};
  if (!p.first || !p.second) return {nullptr, nullptr};
  net->ev_pending.push_back({what, p});
  return p;
}

df_status prof_collect(df_net* net) {
  if (net->ev_pending.empty()) return DF_OK;
  DF_CUDA(cudaStreamSynchronize(net->stream));
  for (auto& pe : net->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) {
      net->prof_ms[pe.first] += ms;
      net->prof_n[pe.first] += 1;
    }
    net->ev_free.push_back(pe.second.first);
    net->ev_free.push_back(pe.second.second);
  }
  net->ev_pending.clear();
  return DF_OK;
}

df_status enqueue_step(df_net* net, bool no_batch, bool capturing = false) {
  cudaStream_t s = net->stream;
  const auto step_ev = prof_pair(net, DF_PROF_STEP, capturing);
  if (step_ev.first) DF_CUDA(cudaEventRecord(step_ev.first, s));
  for (const Op& op : net->program) {
    switch (op.kind) {
      case kOpCopy: {
        const auto ev = prof_pair(net, DF_PROF_COPY_BODY, capturing);
        DF_CUDA(launch_copy(op.copy, net->n_sm, s, ev.first, ev.second));
        break;
      }
      case kOpMd: {
        const auto ev = prof_pair(net, DF_PROF_MD_MAIN, capturing);
        DF_CUDA(launch_md_step(op.md, &op.md_tma, net->n_sm, s, ev.first, ev.second));
        break;
      }
      case kOpDyn:
        DF_CUDA(launch_dyn(op.dyn, net->n_sm, s));
        break;
      case kOpImg:
        DF_CUDA(launch_img(op.img, net->n_sm, s));
        break;
      case kOpDpd: {
        const ActorH& A0 = net->actors[op.dpd_first_actor];
        uint32_t tile = A0.tile, threads = A0.threads;
        if (!tile || !threads) {
          const DpdArgs& a = net->dpd_host[net->dpd_index[op.dpd_first_actor]];
          tile = default_tile(a);
          threads = 256;
        }
        const int n_launch = no_batch ? op.dpd_n : 1;
        const int per = no_batch ? 1 : op.dpd_n;
        for (int i = 0; i < n_launch; ++i) {
          const auto ev = prof_pair(net, DF_PROF_DPD_BODY, capturing);
          // without timing events the plan and body are programmatic dependents
          const bool pdl = !ev.first;
          DF_CUDA(launch_dpd_plan(op.dpd_dev + i, per, s, pdl));
          if (ev.first) DF_CUDA(cudaEventRecord(ev.first, s));
          DF_CUDA(launch_dpd_body(op.dpd_dev + i, no_batch ? nullptr : op.dpd_order, per, tile, threads,
                                  op.max_mt, net->n_sm, s, pdl));
          if (ev.second) DF_CUDA(cudaEventRecord(ev.second, s));
        }
        break;
      }
    }
    for (const SpillArgs& sp : op.spills) DF_CUDA(launch_spill(sp, s));
  }
  if (net->io_used) DF_CUDA(launch_publish(net->d_eng, s));
  if (step_ev.second) DF_CUDA(cudaEventRecord(step_ev.second, s));
  return DF_OK;
}

// Tap-gradient partial sums of df_dpd_backward: one buffer per (device,
// stream), so calls on different streams never share one, and calls on one
// stream are ordered by it.  A buffer that is outgrown is retired, never
// freed while the process runs: kernels already enqueued, and CUDA graphs
// captured earlier, may still write to it.
std::mutex g_scratch_mu;
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, uintptr_t>, Scratch> g_scratch;
std::vector<void*> g_scratch_retired;

}  // namespace

// Device copy of the step program for the persistent kernel.
df_status build_persistent(df_net* net) {
  if (net->d_persist_ops) return DF_OK;
  std::vector<PersistOp> ops;
  size_t bytes = 0;
  for (const Op& op : net->program) {
    if (!op.spills.empty()) bytes += align256(sizeof(SpillArgs) * op.spills.size());
    if (op.kind == kOpCopy) bytes += align256(sizeof(CopyArgs));
    if (op.kind == kOpDyn) bytes += align256(sizeof(DynArgs));
    if (op.kind == kOpMd) bytes += align256(sizeof(MdArgs));
    if (op.kind == kOpImg) bytes += align256(sizeof(ImgArgs));
  }
  bytes += align256(sizeof(PersistOp) * std::max<size_t>(1, 2 * net->program.size()));
  if (cudaMalloc(&net->persist_mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    net->persist_mem = nullptr;
    return DF_ENOMEM;
  }
  uint8_t* base = static_cast<uint8_t*>(net->persist_mem);
  size_t off = 0;
  int max_group = 1, mtmax = 1;
  size_t img_smem = 0;
  // A program of predistorter groups alone whose largest step has no more
  // items (chunks of 256 outputs) than a one-CTA-per-SM grid has warps runs
  // on that grid: its steps are latency bound, and half the CTAs make the
  // launch and every grid barrier cheaper (a 64 x 4096-sample stream through
  // capacity-8 FIFOs: 19.2 -> 17.1 us per step).
  bool dpd_only = true;
  uint64_t max_items = 0;
  for (const Op& op : net->program) {
    PersistOp p{};
    if (op.kind == kOpCopy) {
      DF_CUDA(cudaMemcpyAsync(base + off, &op.copy, sizeof(CopyArgs), cudaMemcpyHostToDevice, net->stream));
      p.kind = kPersistCopy;
      p.args = base + off;
      off += align256(sizeof(CopyArgs));
    } else if (op.kind == kOpDyn) {
      DF_CUDA(cudaMemcpyAsync(base + off, &op.dyn, sizeof(DynArgs), cudaMemcpyHostToDevice, net->stream));
      p.kind = kPersistDyn;
      p.args = base + off;
      off += align256(sizeof(DynArgs));
    } else if (op.kind == kOpMd) {
      DF_CUDA(cudaMemcpyAsync(base + off, &op.md, sizeof(MdArgs), cudaMemcpyHostToDevice, net->stream));
      p.kind = kPersistMd;
      p.args = base + off;
      off += align256(sizeof(MdArgs));
    } else if (op.kind == kOpImg) {
      DF_CUDA(cudaMemcpyAsync(base + off, &op.img, sizeof(ImgArgs), cudaMemcpyHostToDevice, net->stream));
      p.kind = kPersistImg;
      p.args = base + off;
      off += align256(sizeof(ImgArgs));
      if (op.img.kind != DF_THRES) img_smem = std::max(img_smem, img_smem_bytes(op.img.W));
    } else {
      p.kind = kPersistDpd;
      p.n = op.dpd_n;
      p.args = op.dpd_dev;
      p.order = op.dpd_order;
      max_group = std::max(max_group, op.dpd_n);
      mtmax = std::max(mtmax, op.max_mt);
      const int i0 = net->dpd_index[op.dpd_first_actor];
      for (int i = 0; i < op.dpd_n; ++i) {
        const DpdArgs& d = net->dpd_host[i0 + i];
        max_items += (uint64_t)d.n_max * ((d.L + 255) / 256);
      }
    }
    if (op.kind != kOpDpd) dpd_only = false;
    ops.push_back(p);
    if (!op.spills.empty()) {
      DF_CUDA(cudaMemcpyAsync(base + off, op.spills.data(), sizeof(SpillArgs) * op.spills.size(),
                              cudaMemcpyHostToDevice, net->stream));
      PersistOp q{};
      q.kind = kPersistSpill;
      q.n = (int)op.spills.size();
      q.args = base + off;
      off += align256(sizeof(SpillArgs) * op.spills.size());
      ops.push_back(q);
    }
  }
  net->d_persist_ops = reinterpret_cast<PersistOp*>(base + off);
  if (!ops.empty())
    DF_CUDA(cudaMemcpyAsync(net->d_persist_ops, ops.data(), sizeof(PersistOp) * ops.size(),
                            cudaMemcpyHostToDevice, net->stream));
  net->persist_n_ops = (int)ops.size();
  net->persist_mtmax = mtmax <= 16 ? 16 : 32;
  net->persist_smem = std::max(persistent_smem(net->persist_mtmax, max_group), img_smem);
  net->persist_per_sm = dpd_only && max_items <= (uint64_t)net->n_sm * (kPersistThreads / 32) ? 1 : 0;
  DF_CUDA(persistent_prepare(net->persist_smem));
  DF_CUDA(cudaStreamSynchronize(net->stream));
  return DF_OK;
}

df_status cuda_status(cudaError_t e) {
  return e == cudaSuccess ? DF_OK : record_cuda(e, "kernel launch");
}

extern "C" {

const char* df_last_error(void) { return g_last_error; }

const char* df_status_str(df_status s) {
  switch (s) {
    case DF_OK: return "ok";
    case DF_EINVAL: return "invalid argument or network";
    case DF_ENOMEM: return "out of memory";
    case DF_EFULL: return "channel full";
    case DF_EEMPTY: return "channel empty";
    case DF_ESTATE: return "call not allowed in this state";
    case DF_EDEADLOCK: return "no quiescence within the step limit";
    case DF_ETIMEOUT: return "device-side wait timed out";
    case DF_ECUDA: return "CUDA runtime error";
    case DF_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

df_status df_net_create(df_net** out, int device, void* cuda_stream) {
  if (!out) return DF_EINVAL;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return DF_EINVAL;
  std::unique_ptr<df_net> net(new (std::nothrow) df_net());
  if (!net) return DF_ENOMEM;
  net->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  DF_CUDA(cudaGetDeviceProperties(&prop, device));
  net->n_sm = prop.multiProcessorCount;
  if (cuda_stream) {
    net->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    DF_CUDA(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking));
    net->own_stream = true;
  }
  DF_CUDA(cudaMallocHost(reinterpret_cast<void**>(&net->h_pin), 64));
  *out = net.release();
  return DF_OK;
}

void df_net_destroy(df_net* net) {
  if (!net) return;
  DeviceGuard g(net->device);
  if (net->stream) cudaStreamSynchronize(net->stream);
  for (auto& kv : net->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& pe : net->ev_pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t e : net->ev_free) cudaEventDestroy(e);
  if (net->persist_mem) cudaFree(net->persist_mem);
  if (net->arena) cudaFree(net->arena);
  if (net->h_pin) cudaFreeHost(net->h_pin);
  if (net->h_pub) cudaFreeHost(net->h_pub);
  for (int i = 0; i < 2; ++i) {
    if (net->io_stream[i]) {
      cudaStreamSynchronize(net->io_stream[i]);
      cudaStreamDestroy(net->io_stream[i]);
    }
  }
  if (net->own_stream) cudaStreamDestroy(net->stream);
  delete net;
}

df_status df_actor_add(df_net* net, int32_t kind, const void* params, size_t params_bytes,
                       int32_t* out_id) {
  if (!net || !out_id) return DF_EINVAL;
  if (net->finalized) return DF_ESTATE;
  ActorH A;
  A.kind = kind;
  switch (kind) {
    case DF_SOURCE:
    case DF_SINK:
    case DF_COPY:
      break;
    case DF_DPD:
    case DF_DPD_POLY:
    case DF_DPD_FIR:
    case DF_DPD_ADD: {
      if (!params || params_bytes != sizeof(df_dpd_params)) return DF_EINVAL;
      std::memcpy(&A.dpd, params, sizeof(df_dpd_params));
      const df_dpd_params& p = A.dpd;
      if (p.K < 1 || p.K > DF_MAX_BRANCHES || p.M < 1 || p.M > DF_MAX_TAPS) return DF_EINVAL;
      if (p.block_len < 1 || !p.h) return DF_EINVAL;
      for (int k = 0; k < p.K; ++k)
        if (p.orders[k] < 1 || p.orders[k] % 2 == 0 || p.orders[k] > 63) return DF_EINVAL;
      A.h.assign(p.h, p.h + 2 * (size_t)p.K * p.M);
      A.dpd.h = nullptr;
      break;
    }
    case DF_GAUSS5:
    case DF_THRES:
    case DF_MED5: {
      if (!params || params_bytes != sizeof(df_img_params)) return DF_EINVAL;
      std::memcpy(&A.img, params, sizeof(df_img_params));
      const df_img_params& m = A.img;
      if (m.width < 1 || m.height < 1 || m.height > 65536) return DF_EINVAL;
      // valid frames the image kernels do not implement: 16-byte row vectors, 2048-pixel rows
      if (m.width < 16 || m.width % 16 || m.width > kImgMaxWidth) return DF_ENOTSUP;
      if (kind == DF_THRES && (m.threshold < 0 || m.threshold > 255)) return DF_EINVAL;
      break;
    }
    case DF_MD: {
      if (!params || params_bytes != sizeof(df_md_params)) return DF_EINVAL;
      std::memcpy(&A.md, params, sizeof(df_md_params));
      const df_md_params& m = A.md;
      if (m.width < 1 || m.height < 1 || m.tile < 1) return DF_EINVAL;
      if (m.width > 65536 || m.height > 65536 || m.threshold < 0 || m.threshold > 255)
        return DF_EINVAL;
      // valid frames the detector does not implement: 32-pixel row words, 16x16 tiles
      if (m.width % 32 || m.tile != 16) return DF_ENOTSUP;
      break;
    }
    default:
      return DF_EINVAL;
  }
  net->actors.push_back(std::move(A));
  *out_id = (int32_t)net->actors.size() - 1;
  return DF_OK;
}

df_status df_channel_connect(df_net* net, int32_t src_actor, int32_t src_port, int32_t dst_actor,
                             int32_t dst_port, uint32_t token_bytes, uint32_t rate,
                             uint32_t capacity_tokens, uint32_t initial_tokens,
                             const void* initial_data, int32_t* out_ch) {
  if (!net || !out_ch) return DF_EINVAL;
  if (net->finalized) return DF_ESTATE;
  const int na = (int)net->actors.size();
  if (src_actor < 0 || src_actor >= na || dst_actor < 0 || dst_actor >= na) return DF_EINVAL;
  if (src_actor == dst_actor) return DF_EINVAL;
  if (src_port < 0 || dst_port < 0 || src_port >= 64 || dst_port >= 64) return DF_EINVAL;
  if (token_bytes == 0 || rate == 0) return DF_EINVAL;
  ActorH& S = net->actors[src_actor];
  ActorH& D = net->actors[dst_actor];
  const bool eq1 = capacity_tokens == DF_CAPACITY_EQ1;
  if (eq1) {
    // Eq. 1: a double buffer of 2r tokens, or 3r + 1 slots around one delay
    // token of which 3r hold unread tokens (Fig. 2)
    if (initial_tokens > 1 || S.kind == DF_MD || (uint64_t)rate * 3 > 0xffffffffull) return DF_EINVAL;
    capacity_tokens = initial_tokens ? 3 * rate : 2 * rate;
  }
  if ((uint64_t)capacity_tokens < (uint64_t)initial_tokens + rate) return DF_EINVAL;
  if (S.kind == DF_SINK || D.kind == DF_SOURCE) return DF_EINVAL;
  if ((int)S.out.size() > src_port && S.out[src_port] >= 0) return DF_EINVAL;
  if ((int)D.in.size() > dst_port && D.in[dst_port] >= 0) return DF_EINVAL;
  if (is_dynamic(D.kind) && dst_port == 0 && (rate != 1 || initial_tokens != 0 || token_bytes != 4))
    return DF_EINVAL;
  ChanH c{};
  c.src = src_actor; c.sport = src_port; c.dst = dst_actor; c.dport = dst_port;
  c.tok = token_bytes; c.rate = rate; c.cap = capacity_tokens; c.init = initial_tokens;
  c.eq1 = eq1;
  if (initial_tokens && initial_data) {
    const uint8_t* p = static_cast<const uint8_t*>(initial_data);
    c.init_data.assign(p, p + (size_t)initial_tokens * token_bytes);
  }
  const int32_t id = (int32_t)net->chans.size();
  net->chans.push_back(std::move(c));
  if ((int)S.out.size() <= src_port) S.out.resize(src_port + 1, -1);
  if ((int)D.in.size() <= dst_port) D.in.resize(dst_port + 1, -1);
  S.out[src_port] = id;
  D.in[dst_port] = id;
  *out_ch = id;
  return DF_OK;
}

df_status df_net_finalize(df_net* net) {
  if (!net) return DF_EINVAL;
  if (net->finalized) return DF_ESTATE;
  for (int a = 0; a < (int)net->actors.size(); ++a) {
    const df_status st = validate_actor(net, a);
    if (st != DF_OK) return st;
  }
  DeviceGuard g(net->device);
  // ---- arena layout ----
  size_t off = 0;
  auto take = [&](size_t bytes) {
    Piece p;
    p.off = off;
    p.bytes = bytes;
    off += align256(bytes);
    return p;
  };
  std::vector<Piece> ring(net->chans.size());
  for (size_t c = 0; c < net->chans.size(); ++c)
    ring[c] = take((size_t)net->chans[c].slots() * net->chans[c].tok);
  const Piece p_ctr = take(2 * sizeof(uint64_t) * std::max<size_t>(1, net->chans.size()));
  const Piece p_eng = take(sizeof(EngineDev));
  struct DpdPieces { Piece plan, masks, rank, act, prev, cnt, hist, parity, h; };
  struct MdPieces { Piece plan, counts, tot, off; };
  std::vector<DpdPieces> dp;
  std::vector<MdPieces> mp;
  std::vector<Piece> cp;
  net->dpd_index.assign(net->actors.size(), -1);
  std::vector<int> md_index(net->actors.size(), -1), copy_index(net->actors.size(), -1);
  std::vector<Piece> ip;
  std::vector<int> img_index(net->actors.size(), -1);
  struct DynPieces { Piece plan, masks, rank; };
  std::vector<DynPieces> yp;
  std::vector<int> dyn_index(net->actors.size(), -1);
  auto is_dpd_like = [](int kind) { return kind == DF_DPD || kind == DF_DPD_FIR; };
  auto dpd_nmax = [&](const ActorH& A) {
    if (A.kind == DF_DPD_FIR) return std::min(net->chans[A.in[0]].cap, net->chans[A.out[0]].cap);
    return std::min({net->chans[A.in[0]].cap, net->chans[A.in[1]].cap, net->chans[A.out[0]].cap});
  };
  for (int a = 0; a < (int)net->actors.size(); ++a) {
    const ActorH& A = net->actors[a];
    if (A.kind == DF_DPD_POLY || A.kind == DF_DPD_ADD) {
      const uint32_t nmax = net->chans[A.in[0]].cap;
      DynPieces q;
      q.plan = take(sizeof(DynPlanHdr));
      q.masks = take(4ull * nmax);
      q.rank = take(4ull * nmax * (A.dpd.K + 1));
      dyn_index[a] = (int)yp.size();
      yp.push_back(q);
    }
    if (is_dpd_like(A.kind)) {
      const int K = A.kind == DF_DPD_FIR ? 1 : A.dpd.K;
      const int MT = dpd_supported_mt(A.dpd.M);
      const uint32_t nmax = dpd_nmax(A);
      DpdPieces q;
      q.plan = take(sizeof(DpdPlanHdr));
      q.masks = take(4ull * nmax);
      q.rank = take(4ull * nmax * K);
      q.act = take(4ull * nmax * K);
      q.prev = take(4ull * nmax * K);
      q.cnt = take(4ull * K);
      q.hist = take(8ull * 2 * K * std::max(1, MT - 1));
      q.parity = take(4);
      q.h = take(16ull * K * MT);
      net->dpd_index[a] = (int)dp.size();
      dp.push_back(q);
    } else if (A.kind == DF_MD) {
      const uint32_t nmax = std::min({net->chans[A.in[0]].cap, net->chans[A.in[1]].cap,
                                      net->chans[A.out[1]].cap});
      MdPieces q;
      q.plan = take(sizeof(MdPlanHdr));
      q.counts = take(2ull * nmax * tiles_per_frame(A.md));
      q.tot = take(4ull * nmax);
      q.off = take(8ull * (nmax + 1));
      md_index[a] = (int)mp.size();
      mp.push_back(q);
    } else if (A.kind == DF_COPY) {
      copy_index[a] = (int)cp.size();
      cp.push_back(take(sizeof(CopyPlan)));
    } else if (A.kind == DF_GAUSS5 || A.kind == DF_THRES || A.kind == DF_MED5) {
      img_index[a] = (int)ip.size();
      ip.push_back(take(sizeof(ImgPlan)));
    }
  }
  const Piece p_dpd_args = take(sizeof(DpdArgs) * std::max<size_t>(1, dp.size()));
  const Piece p_dpd_order = take(sizeof(uint16_t) * std::max<size_t>(1, dp.size()));
  net->arena_bytes = off;
  if (cudaMalloc(&net->arena, std::max<size_t>(off, 256)) != cudaSuccess) {
    cudaGetLastError();
    net->arena = nullptr;
    return DF_ENOMEM;
  }
  uint8_t* base = net->arena;
  cudaStream_t s = net->stream;
  DF_CUDA(cudaMemsetAsync(base, 0, off, s));
  net->d_ctr = reinterpret_cast<uint64_t*>(base + p_ctr.off);
  net->d_eng = reinterpret_cast<EngineDev*>(base + p_eng.off);
  // ---- channels: descriptors, initial tokens, counters ----
  std::vector<uint64_t> ctr0(2 * net->chans.size(), 0);
  for (size_t c = 0; c < net->chans.size(); ++c) {
    ChanH& C = net->chans[c];
    C.desc.ring = base + ring[c].off;
    C.desc.cap = C.cap;
    C.desc.tok = C.tok;
    C.desc.rate = C.rate;
    C.desc.id = (uint32_t)c;
    C.desc.wshift = 0;
    C.wdesc = C.desc;
    if (C.slots() > C.cap) {            // writers start at slot 1 (Fig. 2)
      C.wdesc.ring += C.tok;
      C.wdesc.wshift = 1;
    }
    if (C.init && !C.init_data.empty())
      DF_CUDA(cudaMemcpyAsync(C.desc.ring, C.init_data.data(), C.init_data.size(),
                              cudaMemcpyHostToDevice, s));
    ctr0[2 * c] = C.init;
  }
  if (!ctr0.empty()) {
    DF_CUDA(cudaMemcpyAsync(net->d_ctr, ctr0.data(), ctr0.size() * 8, cudaMemcpyHostToDevice, s));
  }
  // published counters in mapped host memory: a concurrent push or pop reads
  // them with a plain load, no copy and no wait
  DF_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&net->h_pub),
                        2 * sizeof(uint64_t) * std::max<size_t>(1, net->chans.size()), cudaHostAllocMapped));
  if (!ctr0.empty()) std::memcpy(net->h_pub, ctr0.data(), ctr0.size() * 8);
  DF_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&net->d_pub), net->h_pub, 0));
  net->host_ctr = ctr0;
  {
    // engine word: where the counters and their published copy are
    uint64_t* ptrs[2] = {net->d_ctr, net->d_pub};
    const uint32_t words = (uint32_t)(2 * net->chans.size());
    DF_CUDA(cudaMemcpyAsync(&net->d_eng->ctr, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(&net->d_eng->n_words, &words, sizeof(words), cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaStreamSynchronize(s));
  }
  // ---- per-actor device state and the step program ----
  net->dpd_host.assign(dp.size(), DpdArgs{});
  std::vector<std::vector<float4>> hpad(dp.size());
  net->d_dpd = reinterpret_cast<DpdArgs*>(base + p_dpd_args.off);
  for (int a = 0; a < (int)net->actors.size(); ++a) {
    const ActorH& A = net->actors[a];
    if (is_dpd_like(A.kind)) {
      const bool fir = A.kind == DF_DPD_FIR;
      const int i = net->dpd_index[a];
      const DpdPieces& q = dp[i];
      DpdArgs& d = net->dpd_host[i];
      if (fir) {
        d.ctrl = ChanDesc{};                 // static: every firing has mask 1
        d.data = net->chans[A.in[0]].desc;
      } else {
        d.ctrl = net->chans[A.in[0]].desc;
        d.data = net->chans[A.in[1]].desc;
      }
      d.out = net->chans[A.out[0]].wdesc;
      d.ctr = net->d_ctr;
      d.eng = net->d_eng;
      d.K = fir ? 1 : A.dpd.K;
      d.M = A.dpd.M;
      d.MT = dpd_supported_mt(A.dpd.M);
      d.L = A.dpd.block_len;
      d.n_max = dpd_nmax(A);
      if (fir) d.orders[0] = 1;              // the branch signal arrives already formed
      else
        for (int k = 0; k < A.dpd.K; ++k) d.orders[k] = A.dpd.orders[k];
      d.plan = reinterpret_cast<DpdPlanHdr*>(base + q.plan.off);
      d.masks = reinterpret_cast<uint32_t*>(base + q.masks.off);
      d.rank = reinterpret_cast<uint32_t*>(base + q.rank.off);
      d.act = reinterpret_cast<uint32_t*>(base + q.act.off);
      d.prev = reinterpret_cast<int32_t*>(base + q.prev.off);
      d.cnt = reinterpret_cast<uint32_t*>(base + q.cnt.off);
      d.hist = reinterpret_cast<float2*>(base + q.hist.off);
      d.parity = reinterpret_cast<uint32_t*>(base + q.parity.off);
      // taps as {hx, hx, hy, hy}: the body's two-lane FMAs take {hx, hx} and
      // {hy, hy} straight from one 16-byte load
      float4* hd = reinterpret_cast<float4*>(base + q.h.off);
      d.h = hd;
      hpad[i].assign((size_t)d.K * d.MT, make_float4(0.f, 0.f, 0.f, 0.f));
      for (int k = 0; k < d.K; ++k) {
        const size_t row = fir ? (size_t)A.dpd.branch : (size_t)k;
        for (int m = 0; m < d.M; ++m) {
          const float hx = A.h[2 * (row * d.M + m)], hy = A.h[2 * (row * d.M + m) + 1];
          hpad[i][(size_t)k * d.MT + m] = make_float4(hx, hx, hy, hy);
        }
      }
      DF_CUDA(cudaMemcpyAsync(hd, hpad[i].data(), hpad[i].size() * sizeof(float4),
                              cudaMemcpyHostToDevice, s));
    }
  }
  if (!net->dpd_host.empty())
    DF_CUDA(cudaMemcpyAsync(net->d_dpd, net->dpd_host.data(), sizeof(DpdArgs) * net->dpd_host.size(),
                            cudaMemcpyHostToDevice, s));
  net->program.clear();
  // Fig. 2 copy after the writer of a delay channel in the paper's layout
  auto add_spill = [&](Op& op, int32_t ch, const uint64_t* wr_before) {
    const ChanH& C = net->chans[ch];
    if (!C.wdesc.wshift) return;
    SpillArgs sp{};
    sp.ring = C.desc.ring;
    sp.cap = C.cap;
    sp.tok = C.tok;
    sp.wr_before = wr_before;
    sp.ctr = net->d_ctr;
    sp.id = (uint32_t)ch;
    sp.unit = C.tok % 16 == 0 ? 16 : (C.tok % 4 == 0 ? 4 : 1);
    op.spills.push_back(sp);
  };
  std::vector<int> group;                 // current predistorter group (actor ids)
  std::vector<std::vector<uint16_t>> host_orders;
  std::vector<std::pair<uint16_t*, size_t>> order_copies;
  auto flush_group = [&]() {
    if (group.empty()) return;
    Op op{};
    op.kind = kOpDpd;
    for (int a : group) add_spill(op, net->actors[a].out[0], &net->dpd_host[net->dpd_index[a]].plan->wr_out0);
    op.dpd_dev = net->d_dpd + net->dpd_index[group[0]];
    op.dpd_n = (int)group.size();
    op.dpd_first_actor = group[0];
    for (int a : group) op.max_mt = std::max(op.max_mt, net->dpd_host[net->dpd_index[a]].MT);
    // the body lays out its items actor by actor in this order: equal padded
    // tap counts together (stable), so neighbouring items share kernel code
    std::vector<uint16_t> ord(group.size());
    for (size_t j = 0; j < ord.size(); ++j) ord[j] = (uint16_t)j;
    std::stable_sort(ord.begin(), ord.end(), [&](uint16_t x, uint16_t y) {
      return net->dpd_host[net->dpd_index[group[x]]].MT < net->dpd_host[net->dpd_index[group[y]]].MT;
    });
    host_orders.push_back(std::move(ord));
    uint16_t* od = reinterpret_cast<uint16_t*>(base + p_dpd_order.off) + net->dpd_index[group[0]];
    order_copies.push_back({od, host_orders.size() - 1});
    op.dpd_order = od;
    net->program.push_back(op);
    group.clear();
  };
  auto linked = [&](int a, int b) {
    for (const ChanH& c : net->chans)
      if ((c.src == a && c.dst == b) || (c.src == b && c.dst == a)) return true;
    return false;
  };
  for (int a = 0; a < (int)net->actors.size(); ++a) {
    const ActorH& A = net->actors[a];
    // host endpoints never fire inside a step, so they do not split a group
    if (A.kind == DF_SOURCE || A.kind == DF_SINK) continue;
    if (!is_dpd_like(A.kind)) flush_group();
    if (A.kind == DF_DPD_POLY || A.kind == DF_DPD_ADD) {
      Op op{};
      op.kind = kOpDyn;
      DynArgs& y = op.dyn;
      const DynPieces& q = yp[dyn_index[a]];
      const bool poly = A.kind == DF_DPD_POLY;
      y.kind = A.kind;
      y.K = A.dpd.K;
      for (int k = 0; k < A.dpd.K; ++k) y.orders[k] = A.dpd.orders[k];
      y.L = A.dpd.block_len;
      y.ctrl = net->chans[A.in[0]].desc;
      y.np = A.dpd.K + 1;
      for (int p = 0; p < y.np; ++p) {
        const bool always = poly ? p == 0 : p == A.dpd.K;
        y.bit[p] = always ? -1 : (poly ? p - 1 : p);
        y.is_out[p] = poly ? (p > 0) : (p == A.dpd.K);
        const int32_t c = poly ? (p == 0 ? A.in[1] : A.out[p - 1]) : (p < A.dpd.K ? A.in[p + 1] : A.out[0]);
        y.port[p] = y.is_out[p] ? net->chans[c].wdesc : net->chans[c].desc;
      }
      y.n_max = net->chans[A.in[0]].cap;
      y.ctr = net->d_ctr;
      y.eng = net->d_eng;
      y.plan = reinterpret_cast<DynPlanHdr*>(base + q.plan.off);
      y.masks = reinterpret_cast<uint32_t*>(base + q.masks.off);
      y.rank = reinterpret_cast<uint32_t*>(base + q.rank.off);
      for (int p = 0; p < y.np; ++p)
        if (y.is_out[p]) add_spill(op, poly ? A.out[p - 1] : A.out[0], &y.plan->base[p]);
      net->program.push_back(op);
    } else if (is_dpd_like(A.kind)) {
      bool ok = (int)group.size() < 1024;
      for (int b : group) ok = ok && !linked(a, b);
      if (!ok) flush_group();
      group.push_back(a);
    } else if (A.kind == DF_COPY) {
      Op op{};
      op.kind = kOpCopy;
      CopyArgs& c = op.copy;
      c.in = net->chans[A.in[0]].desc;
      c.n_out = (int)A.out.size();
      int unit = 16;
      auto fit = [&](uint64_t tok) {
        while (unit > 1 && tok % unit) unit = unit == 16 ? 4 : 1;
      };
      fit(c.in.tok);
      for (int p = 0; p < c.n_out; ++p) {
        c.out[p] = net->chans[A.out[p]].wdesc;
        fit(c.out[p].tok);
      }
      c.unit = unit;
      c.ctr = net->d_ctr;
      c.eng = net->d_eng;
      c.plan = reinterpret_cast<CopyPlan*>(base + cp[copy_index[a]].off);
      for (int p = 0; p < c.n_out; ++p) add_spill(op, A.out[p], &c.plan->wr0[p]);
      net->program.push_back(op);
    } else if (A.kind == DF_GAUSS5 || A.kind == DF_THRES || A.kind == DF_MED5) {
      Op op{};
      op.kind = kOpImg;
      ImgArgs& m = op.img;
      m.kind = A.kind;
      m.n_in = (int)A.in.size();
      for (int i = 0; i < m.n_in; ++i) m.in[i] = net->chans[A.in[i]].desc;
      m.n_out = (int)A.out.size();
      for (int p = 0; p < m.n_out; ++p) m.out[p] = net->chans[A.out[p]].wdesc;
      m.W = A.img.width;
      m.H = A.img.height;
      m.thr = A.img.threshold;
      if (A.kind == DF_THRES) {
        // Both inputs come from one writer that puts the same tokens on all its
        // outputs, the second with one delay token: then within a step the
        // previous frame of window frame j >= 1 is frame j - 1 of the first input.
        const ChanH &cur = net->chans[A.in[0]], &prev = net->chans[A.in[1]];
        const int wk = net->actors[cur.src].kind;
        const bool broadcast = wk == DF_SOURCE || wk == DF_COPY || wk == DF_GAUSS5 || wk == DF_THRES ||
                               wk == DF_MED5;
        m.dedup = (cur.src == prev.src && broadcast && cur.init == 0 && prev.init == 1) ? 1 : 0;
      }
      if (A.kind == DF_MED5) {
        // Thres writes only 0 and 255: with such initial tokens too, the
        // median of five is a bitwise majority without a per-band check
        const ChanH& in = net->chans[A.in[0]];
        bool bin = net->actors[in.src].kind == DF_THRES;
        for (uint8_t v : in.init_data) bin = bin && (v == 0 || v == 255);
        m.binary_in = bin ? 1 : 0;
      }
      m.wait_limit_ns = net->wait_limit_ns;
      m.ctr = net->d_ctr;
      m.eng = net->d_eng;
      m.plan = reinterpret_cast<ImgPlan*>(base + ip[img_index[a]].off);
      for (int p = 0; p < m.n_out; ++p) add_spill(op, A.out[p], &m.plan->wr0[p]);
      net->program.push_back(op);
    } else if (A.kind == DF_MD) {
      Op op{};
      op.kind = kOpMd;
      MdArgs& m = op.md;
      const MdPieces& q = mp[md_index[a]];
      const ChanH &cur = net->chans[A.in[0]], &prev = net->chans[A.in[1]];
      m.cur = cur.desc;
      m.prev = prev.desc;
      m.rec = net->chans[A.out[0]].desc;
      m.cnt = net->chans[A.out[1]].desc;
      m.ctr = net->d_ctr;
      m.eng = net->d_eng;
      m.W = A.md.width;
      m.H = A.md.height;
      m.thr = A.md.threshold;
      m.words = m.W / 32;
      m.tiles_x = (m.W + 15) / 16;
      m.tiles_y = (m.H + 15) / 16;
      m.n_tiles = m.tiles_x * m.tiles_y;
      m.strips = (m.H + 15) / 16;
      // The previous-frame channel carries the current-frame stream delayed by
      // exactly one token when both come from the same source broadcast, the
      // current channel has no initial token and the previous channel one.
      m.dedup = (cur.src == prev.src && net->actors[cur.src].kind == DF_SOURCE &&
                 cur.init == 0 && prev.init == 1) ? 1 : 0;
      m.shared_rows = (m.dedup && (uint64_t)cur.cap * cur.tok < (1ull << 31)) ? 1 : 0;
      m.n_max = std::min({cur.cap, prev.cap, net->chans[A.out[1]].cap});
      m.plan = reinterpret_cast<MdPlanHdr*>(base + q.plan.off);
      m.counts = reinterpret_cast<uint16_t*>(base + q.counts.off);
      m.frame_tot = reinterpret_cast<uint32_t*>(base + q.tot.off);
      m.frame_off = reinterpret_cast<uint64_t*>(base + q.off.off);
      m.wait_limit_ns = net->wait_limit_ns;
      if (md_smem_bytes(m.W) > 227 * 1024) return DF_ENOTSUP;
      net->program.push_back(op);
    }
  }
  flush_group();
  for (const auto& oc : order_copies)
    DF_CUDA(cudaMemcpyAsync(oc.first, host_orders[oc.second].data(), host_orders[oc.second].size() * sizeof(uint16_t),
                            cudaMemcpyHostToDevice, s));
  DF_CUDA(cudaStreamSynchronize(s));
  if (!dp.empty()) DF_CUDA(dpd_prepare());  // also covers branch FIR actors
  for (const Op& op : net->program)
    if (op.kind == kOpImg) {
      DF_CUDA(img_prepare());
      break;
    }
  for (Op& op : net->program)
    if (op.kind == kOpMd) {
      DF_CUDA(md_prepare(op.md.W));
      DF_CUDA(md_tma_prepare(op.md, &op.md_tma));
    }
  DF_CUDA(cudaStreamSynchronize(s));
  net->finalized = true;
  return DF_OK;
}

namespace {

// Counters of a channel for a push (writer) or pop (reader) beside running
// steps: the caller's own counter from the host's record (only the host moves
// it), the other side's from the copy published after the last finished step
// (mapped host memory, read with a plain load).
df_status read_io_counters(df_net* net, int32_t ch, bool writer, uint64_t* wr, uint64_t* rd) {
  const volatile uint64_t* pub = net->h_pub;
  *wr = writer ? net->host_ctr[2 * ch] : pub[2 * ch];
  *rd = writer ? pub[2 * ch + 1] : net->host_ctr[2 * ch + 1];
  return DF_OK;
}

// Pinned staging of the calling thread (freed when the thread ends).
struct ThreadPin {
  uint64_t* p = nullptr;
  ~ThreadPin() {
    if (p) cudaFreeHost(p);
  }
};
thread_local ThreadPin t_pin;

// Stream of concurrent pushes (which = 0) or pops (1) and the caller's staging.
df_status io_channel(df_net* net, int which, cudaStream_t* s, uint64_t** pin) {
  if (!t_pin.p) DF_CUDA(cudaMallocHost(&t_pin.p, 64));
  std::lock_guard<std::mutex> lk(net->io_mu);
  net->io_used = true;
  if (!net->io_stream[which])
    DF_CUDA(cudaStreamCreateWithFlags(&net->io_stream[which], cudaStreamNonBlocking));
  *s = net->io_stream[which];
  *pin = t_pin.p;
  return DF_OK;
}

// Push on stream s.  The free space comes from a snapshot of the counters: on
// a concurrent stream the consumer may have read more since, so the snapshot
// only understates it.  The tokens are copied first and wr advanced after
// them on the same stream, so a plan that sees the new wr sees the data.
df_status push_on(df_net* net, int32_t src_actor, const void* src, uint64_t n_tokens,
                  uint64_t* n_pushed, cudaStream_t s, uint64_t* pin) {
  if (!net || (!src && n_tokens)) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  if (src_actor < 0 || src_actor >= (int)net->actors.size()) return DF_EINVAL;
  const ActorH& A = net->actors[src_actor];
  if (A.kind != DF_SOURCE) return DF_EINVAL;
  DeviceGuard g(net->device);
  const bool concurrent = s != net->stream;
  std::vector<uint64_t> wr(A.out.size());
  for (size_t p = 0; p < A.out.size(); ++p) {
    uint64_t w, r;
    const df_status st = concurrent ? read_io_counters(net, A.out[p], true, &w, &r)
                                    : read_counters(net, A.out[p], &w, &r, s, pin);
    if (st != DF_OK) return st;
    if (net->chans[A.out[p]].eq1 && n_tokens % net->chans[A.out[p]].rate) return DF_EINVAL;
    if (net->chans[A.out[p]].cap - (w - r) < n_tokens) return DF_EFULL;
    wr[p] = w;
  }
  if (n_tokens) {
    for (size_t p = 0; p < A.out.size(); ++p) {
      const ChanH& C = net->chans[A.out[p]];
      const ChanDesc& c = C.wdesc;
      if (p > 0 && c.tok == net->chans[A.out[0]].desc.tok) {
        // further broadcast copies come from the first channel (device to device;
        // its reader view, whose Fig. 2 copy is already done)
        const ChanDesc& c0 = net->chans[A.out[0]].desc;
        for (uint64_t done = 0; done < n_tokens;) {
          const uint64_t s0 = (wr[0] + done) % c0.cap, s1 = (wr[p] + done - c.wshift) % c.cap;
          const uint64_t run = std::min({n_tokens - done, c0.cap - s0, c.cap - s1});
          DF_CUDA(cudaMemcpyAsync(c.ring + s1 * c.tok, c0.ring + s0 * c0.tok, run * c.tok,
                                  cudaMemcpyDeviceToDevice, s));
          done += run;
        }
      } else {
        const df_status st = ring_copy(net, c, wr[p], const_cast<void*>(src), n_tokens, true, s);
        if (st != DF_OK) return st;
      }
      // Fig. 2: the token that landed in slot cap is copied to slot 0
      if (c.wshift && (wr[p] - 1) / C.cap != (wr[p] + n_tokens - 1) / C.cap)
        DF_CUDA(cudaMemcpyAsync(C.desc.ring, C.desc.ring + (uint64_t)C.cap * C.tok, C.tok,
                                cudaMemcpyDeviceToDevice, s));
      DF_CUDA(launch_set_u64(net->d_ctr + 2 * A.out[p], wr[p] + n_tokens, s));
    }
    DF_CUDA(cudaStreamSynchronize(s));
    for (size_t p = 0; p < A.out.size(); ++p) net->host_ctr[2 * A.out[p]] = wr[p] + n_tokens;
  }
  if (n_pushed) *n_pushed = n_tokens;
  return DF_OK;
}

// Pop on stream s (snapshot of wr: a concurrent producer may have written
// more since); rd advances after the copy on the same stream.
df_status pop_on(df_net* net, int32_t sink_actor, void* dst, uint64_t max_tokens,
                 uint64_t* n_popped, cudaStream_t s, uint64_t* pin) {
  if (!net || (!dst && max_tokens)) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  if (sink_actor < 0 || sink_actor >= (int)net->actors.size()) return DF_EINVAL;
  const ActorH& A = net->actors[sink_actor];
  if (A.kind != DF_SINK) return DF_EINVAL;
  DeviceGuard g(net->device);
  const int32_t ch = A.in[0];
  uint64_t w, r;
  df_status st = s != net->stream ? read_io_counters(net, ch, false, &w, &r)
                                  : read_counters(net, ch, &w, &r, s, pin);
  if (st != DF_OK) return st;
  const uint64_t n = std::min(max_tokens, w - r);
  if (n) {
    st = ring_copy(net, net->chans[ch].desc, r, dst, n, false, s);
    if (st != DF_OK) return st;
    DF_CUDA(launch_set_u64(net->d_ctr + 2 * ch + 1, r + n, s));
    DF_CUDA(cudaStreamSynchronize(s));
    net->host_ctr[2 * ch + 1] = r + n;
  }
  if (n_popped) *n_popped = n;
  return DF_OK;
}

}  // namespace

df_status df_push(df_net* net, int32_t src_actor, const void* src, uint64_t n_tokens,
                  uint64_t* n_pushed) {
  if (!net) return DF_EINVAL;
  return push_on(net, src_actor, src, n_tokens, n_pushed, net->stream, net->h_pin);
}

df_status df_push_ex(df_net* net, int32_t src_actor, const void* src, uint64_t n_tokens,
                     uint32_t flags, uint64_t* n_pushed) {
  if (!net || (flags & ~(uint32_t)DF_IO_CONCURRENT)) return DF_EINVAL;
  if (!(flags & DF_IO_CONCURRENT)) return df_push(net, src_actor, src, n_tokens, n_pushed);
  if (!net->finalized) return DF_ESTATE;
  cudaStream_t s;
  uint64_t* pin;
  const df_status st = io_channel(net, 0, &s, &pin);
  if (st != DF_OK) return st;
  return push_on(net, src_actor, src, n_tokens, n_pushed, s, pin);
}

df_status df_run_ex(df_net* net, int64_t n_steps, uint32_t flags, uint64_t* n_firings) {
  if (!net) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  if ((flags & DF_RUN_PERSISTENT) && (flags & DF_RUN_NO_BATCH)) return DF_ENOTSUP;
  DeviceGuard g(net->device);
  const bool no_batch = flags & DF_RUN_NO_BATCH;
  uint64_t before = 0;
  if (!(flags & DF_RUN_ASYNC)) {
    if (!net->fired_known) {
      int32_t dst;
      const df_status e = read_engine(net, &before, &dst);
      if (e != DF_OK) return e;
    }
    before = net->fired_seen;
    net->fired_known = false;         // until the run's own read at its end
  } else if (n_steps < 0) {
    return DF_EINVAL;
  } else {
    net->fired_known = false;
  }
  if (flags & DF_RUN_PERSISTENT) {
    df_status st = build_persistent(net);
    if (st != DF_OK) return st;
    const bool publish = net->io_used;
    if (flags & DF_RUN_GRAPH) {
      // one graph holding the persistent launch (its n_steps, or until
      // quiescent); it publishes the counters once concurrent I/O is in use
      auto key = std::make_pair(n_steps, 0x200u | (publish ? 0x100u : 0u));
      auto it = net->graphs.find(key);
      if (it == net->graphs.end()) {
        cudaGraph_t graph;
        DF_CUDA(cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = launch_persistent(net->d_persist_ops, net->persist_n_ops, net->d_eng, n_steps,
                                                 net->wait_limit_ns, net->persist_mtmax, net->persist_smem,
                                                 net->n_sm, net->persist_per_sm, publish, net->stream);
        const cudaError_t ce = cudaStreamEndCapture(net->stream, &graph);
        DF_CUDA(le);
        DF_CUDA(ce);
        cudaGraphExec_t exec;
        DF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        cudaGraphDestroy(graph);
        it = net->graphs.emplace(key, exec).first;
      }
      DF_CUDA(cudaGraphLaunch(it->second, net->stream));
    } else {
      const auto ev = prof_pair(net, DF_PROF_STEP, false);
      if (ev.first) DF_CUDA(cudaEventRecord(ev.first, net->stream));
      DF_CUDA(launch_persistent(net->d_persist_ops, net->persist_n_ops, net->d_eng, n_steps,
                                net->wait_limit_ns, net->persist_mtmax, net->persist_smem, net->n_sm,
                                net->persist_per_sm, publish, net->stream));
      if (ev.second) DF_CUDA(cudaEventRecord(ev.second, net->stream));
    }
  } else if (n_steps >= 0) {
    if (flags & DF_RUN_GRAPH) {
      // the graph of a step ends with the counter publication once concurrent I/O is in use
      auto key = std::make_pair(n_steps, (flags & DF_RUN_NO_BATCH) | (net->io_used ? 0x100u : 0u));
      auto it = net->graphs.find(key);
      if (it == net->graphs.end()) {
        cudaGraph_t graph;
        DF_CUDA(cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
        df_status st = DF_OK;
        for (int64_t i = 0; i < n_steps && st == DF_OK; ++i) st = enqueue_step(net, no_batch, true);
        const cudaError_t ce = cudaStreamEndCapture(net->stream, &graph);
        if (st != DF_OK) return st;
        DF_CUDA(ce);
        cudaGraphExec_t exec;
        DF_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        cudaGraphDestroy(graph);
        it = net->graphs.emplace(key, exec).first;
      }
      DF_CUDA(cudaGraphLaunch(it->second, net->stream));
    } else {
      for (int64_t i = 0; i < n_steps; ++i) {
        const df_status st = enqueue_step(net, no_batch);
        if (st != DF_OK) return st;
      }
    }
  } else {
    // a step fired nothing when the (monotonic) firing total did not move
    const int64_t kMaxSteps = 1 << 20;
    int64_t i = 0;
    uint64_t total = before;
    for (; i < kMaxSteps; ++i) {
      const df_status st = enqueue_step(net, no_batch);
      if (st != DF_OK) return st;
      DF_CUDA(cudaMemcpyAsync(net->h_pin, &net->d_eng->fired_total, 8, cudaMemcpyDeviceToHost,
                              net->stream));
      DF_CUDA(cudaStreamSynchronize(net->stream));
      if (net->h_pin[0] == total) break;
      total = net->h_pin[0];
    }
    if (i == kMaxSteps) return DF_EDEADLOCK;
  }
  if (flags & DF_RUN_ASYNC) return DF_OK;
  uint64_t after = 0;
  int32_t dst = DF_OK;
  const df_status e = read_engine(net, &after, &dst);
  if (e != DF_OK) return e;
  if (dst != DF_OK) return dst;
  if (n_firings) *n_firings = after - before;
  return DF_OK;
}

df_status df_run(df_net* net, int64_t n_steps, uint64_t* n_firings) {
  return df_run_ex(net, n_steps, 0, n_firings);
}

df_status df_sync(df_net* net, uint64_t* total_firings) {
  if (!net) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  DeviceGuard g(net->device);
  uint64_t total = 0;
  int32_t dst = DF_OK;
  const df_status e = read_engine(net, &total, &dst);
  if (e != DF_OK) return e;
  if (dst != DF_OK) return dst;
  if (total_firings) *total_firings = total;
  return DF_OK;
}

df_status df_pop(df_net* net, int32_t sink_actor, void* dst, uint64_t max_tokens,
                 uint64_t* n_popped) {
  if (!net) return DF_EINVAL;
  return pop_on(net, sink_actor, dst, max_tokens, n_popped, net->stream, net->h_pin);
}

df_status df_pop_ex(df_net* net, int32_t sink_actor, void* dst, uint64_t max_tokens, uint32_t flags,
                    uint64_t* n_popped) {
  if (!net || (flags & ~(uint32_t)DF_IO_CONCURRENT)) return DF_EINVAL;
  if (!(flags & DF_IO_CONCURRENT)) return df_pop(net, sink_actor, dst, max_tokens, n_popped);
  if (!net->finalized) return DF_ESTATE;
  cudaStream_t s;
  uint64_t* pin;
  const df_status st = io_channel(net, 1, &s, &pin);
  if (st != DF_OK) return st;
  return pop_on(net, sink_actor, dst, max_tokens, n_popped, s, pin);
}

}  // extern "C"

namespace {

// Events of a streamed run: every push, pop and firing step bumps the
// generation, and a thread with nothing to do sleeps until it moves (or a
// short timeout passes, as a copy on another stream may have freed space).
struct StreamHub {
  std::mutex mu;
  std::condition_variable cv;
  std::atomic<uint64_t> gen{0};
  std::atomic<int32_t> err{DF_OK};
  std::atomic<bool> finished{false};
  std::atomic<int> producers_left{0};
  void bump() {
    {
      std::lock_guard<std::mutex> lk(mu);
      gen.fetch_add(1);
    }
    cv.notify_all();
  }
  uint64_t now() { return gen.load(); }
  bool moved(uint64_t seen) { return gen.load() != seen || err.load() != DF_OK || finished.load(); }
  // A handoff is usually a few microseconds away: spin that long first, then
  // sleep on the condition variable.
  void wait(uint64_t seen) {
    const auto t0 = std::chrono::steady_clock::now();
    while (std::chrono::steady_clock::now() - t0 < std::chrono::microseconds(30))
      if (moved(seen)) return;
    std::unique_lock<std::mutex> lk(mu);
    cv.wait_for(lk, std::chrono::microseconds(200), [&] { return moved(seen); });
  }
  void fail(int32_t st) {
    int32_t ok = DF_OK;
    err.compare_exchange_strong(ok, st);
    bump();
  }
};

uint64_t endpoint_token_bytes(const df_net* net, int32_t actor, int kind) {
  if (actor < 0 || actor >= (int)net->actors.size()) return 0;
  const ActorH& A = net->actors[actor];
  if (A.kind != kind) return 0;
  const std::vector<int32_t>& ports = kind == DF_SOURCE ? A.out : A.in;
  return ports.empty() ? 0 : net->chans[ports[0]].tok;
}

void stream_produce(df_net* net, const df_feed& f, uint64_t tok, StreamHub& hub) {
  const uint8_t* src = static_cast<const uint8_t*>(f.data);
  for (uint64_t done = 0; done < f.n_tokens && hub.err.load() == DF_OK;) {
    const uint64_t n = std::min(f.batch, f.n_tokens - done);
    const uint64_t seen = hub.now();
    const df_status st = df_push_ex(net, f.source, src + done * tok, n, DF_IO_CONCURRENT, nullptr);
    if (st == DF_OK) {
      done += n;
      hub.bump();
    } else if (st == DF_EFULL) {
      hub.wait(seen);
    } else {
      hub.fail(st);
    }
  }
  hub.producers_left.fetch_sub(1);
  hub.bump();
}

void stream_consume(df_net* net, df_drain& d, uint64_t tok, StreamHub& hub) {
  uint8_t* dst = static_cast<uint8_t*>(d.data);
  uint64_t got = 0;
  while (hub.err.load() == DF_OK && got < d.max_tokens) {
    const uint64_t seen = hub.now();
    const bool last = hub.finished.load();     // read before the pop: nothing arrives after it
    uint64_t n = 0;
    const df_status st = df_pop_ex(net, d.sink, dst + got * tok, std::min(d.batch, d.max_tokens - got),
                                   DF_IO_CONCURRENT, &n);
    if (st != DF_OK) {
      hub.fail(st);
      break;
    }
    if (n) {
      got += n;
      hub.bump();
    } else if (last) {
      break;
    } else {
      hub.wait(seen);
    }
  }
  d.n_popped = got;
}

}  // namespace

extern "C" {

df_status df_stream(df_net* net, const df_feed* feeds, int32_t n_feeds, df_drain* drains, int32_t n_drains,
                    uint32_t run_flags, int64_t idle_limit_ns, uint64_t* n_steps) {
  if (!net || n_feeds < 0 || n_drains < 0 || (n_feeds && !feeds) || (n_drains && !drains)) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  if (run_flags & DF_RUN_ASYNC) return DF_EINVAL;
  std::vector<uint64_t> ftok(n_feeds), dtok(n_drains);
  for (int i = 0; i < n_feeds; ++i) {
    ftok[i] = endpoint_token_bytes(net, feeds[i].source, DF_SOURCE);
    if (!ftok[i] || !feeds[i].batch || (!feeds[i].data && feeds[i].n_tokens)) return DF_EINVAL;
  }
  for (int i = 0; i < n_drains; ++i) {
    dtok[i] = endpoint_token_bytes(net, drains[i].sink, DF_SINK);
    if (!dtok[i] || !drains[i].batch || (!drains[i].data && drains[i].max_tokens)) return DF_EINVAL;
  }
  if (idle_limit_ns <= 0) idle_limit_ns = 2000000000LL;
  net->io_used = true;                       // every step publishes its counters
  StreamHub hub;
  hub.producers_left = n_feeds;
  std::vector<std::thread> threads;
  try {
    threads.reserve((size_t)n_feeds + (size_t)n_drains);
    for (int i = 0; i < n_feeds; ++i)
      threads.emplace_back(stream_produce, net, std::cref(feeds[i]), ftok[i], std::ref(hub));
    for (int i = 0; i < n_drains; ++i)
      threads.emplace_back(stream_consume, net, std::ref(drains[i]), dtok[i], std::ref(hub));
  } catch (...) {                            // no thread: stop the ones started, report it
    hub.fail(DF_ENOMEM);
    hub.finished = true;
    hub.bump();
    for (std::thread& t : threads) t.join();
    return DF_ENOMEM;
  }
  // this thread runs the GPU actors: one step at a time, sleeping while
  // nothing can fire; the run is over when the sources are exhausted, a step
  // fired nothing, every drained sink is empty and one more step (after the
  // pops that emptied them) fires nothing either
  uint64_t steps = 0;
  auto idle_since = std::chrono::steady_clock::now();
  while (hub.err.load() == DF_OK) {
    const uint64_t seen = hub.now();
    uint64_t fired = 0;
    const df_status st = df_run_ex(net, 1, run_flags, &fired);
    ++steps;
    if (st != DF_OK) {
      hub.fail(st);
      break;
    }
    if (fired) {
      hub.bump();
      idle_since = std::chrono::steady_clock::now();
      continue;
    }
    if (hub.producers_left.load() == 0) {
      bool empty = true;
      for (int i = 0; i < n_drains && empty; ++i) {
        uint64_t occ = 0;
        const df_status cs = df_channel_counters(net, net->actors[drains[i].sink].in[0], nullptr, nullptr, &occ);
        if (cs != DF_OK) {
          hub.fail(cs);
          break;
        }
        empty = occ == 0;
      }
      if (hub.err.load() != DF_OK) break;
      if (empty) {
        const df_status st2 = df_run_ex(net, 1, run_flags, &fired);
        ++steps;
        if (st2 != DF_OK) {
          hub.fail(st2);
          break;
        }
        if (!fired) break;
        hub.bump();
        continue;
      }
    }
    if (hub.now() == seen) {
      if (std::chrono::steady_clock::now() - idle_since > std::chrono::nanoseconds(idle_limit_ns)) {
        hub.fail(DF_EDEADLOCK);              // nothing moved: a full undrained sink or a cycle
        break;
      }
      hub.wait(seen);
    } else {
      idle_since = std::chrono::steady_clock::now();
    }
  }
  hub.finished = true;
  hub.bump();
  for (std::thread& t : threads) t.join();
  if (hub.err.load() != DF_OK) return hub.err.load();
  if (n_steps) *n_steps = steps;
  return DF_OK;
}

df_status df_channel_counters(df_net* net, int32_t ch, uint64_t* produced, uint64_t* consumed,
                              uint64_t* occupancy) {
  if (!net || ch < 0 || ch >= (int)net->chans.size()) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  DeviceGuard g(net->device);
  uint64_t w, r;
  const df_status st = read_counters(net, ch, &w, &r);
  if (st != DF_OK) return st;
  if (produced) *produced = w - net->chans[ch].init;
  if (consumed) *consumed = r;
  if (occupancy) *occupancy = w - r;
  return DF_OK;
}

df_status df_channel_info(df_net* net, int32_t ch, df_channel_info_t* out) {
  if (!net || !out || ch < 0 || ch >= (int)net->chans.size()) return DF_EINVAL;
  const ChanH& C = net->chans[ch];
  df_channel_info_t i{};
  i.capacity = C.cap;
  i.slots = C.slots();
  i.buffer_bytes = C.slots() * C.tok;
  i.token_bytes = C.tok;
  i.rate = C.rate;
  i.initial_tokens = C.init;
  i.layout = C.eq1 ? DF_LAYOUT_EQ1 : DF_LAYOUT_RING;
  *out = i;
  return DF_OK;
}

df_status df_channel_peek_slots(df_net* net, int32_t ch, uint64_t first_slot, uint64_t n_slots,
                                void* dst) {
  if (!net || ch < 0 || ch >= (int)net->chans.size() || (!dst && n_slots)) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  const ChanH& C = net->chans[ch];
  if (first_slot > C.slots() || n_slots > C.slots() - first_slot) return DF_EINVAL;
  if (!n_slots) return DF_OK;
  DeviceGuard g(net->device);
  DF_CUDA(cudaMemcpyAsync(dst, C.desc.ring + first_slot * C.tok, n_slots * C.tok, cudaMemcpyDeviceToHost,
                          net->stream));
  DF_CUDA(cudaStreamSynchronize(net->stream));
  return DF_OK;
}

df_status df_set_wait_limit(df_net* net, int64_t limit_ns) {
  if (!net || limit_ns <= 0) return DF_EINVAL;
  net->wait_limit_ns = limit_ns;
  for (Op& op : net->program)
    if (op.kind == kOpMd) op.md.wait_limit_ns = limit_ns;
    else if (op.kind == kOpImg) op.img.wait_limit_ns = limit_ns;
  // captured graphs and the persistent kernel's program hold the old limit
  DeviceGuard g(net->device);
  DF_CUDA(cudaStreamSynchronize(net->stream));
  for (auto& kv : net->graphs) cudaGraphExecDestroy(kv.second);
  net->graphs.clear();
  if (net->persist_mem) {
    DF_CUDA(cudaFree(net->persist_mem));
    net->persist_mem = nullptr;
    net->d_persist_ops = nullptr;
  }
  return DF_OK;
}

df_status df_selftest_wait_timeout(df_net* net, int64_t limit_ns) {
  if (!net || limit_ns <= 0) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  DeviceGuard g(net->device);
  df_status st = fail_if_device_error(net);
  if (st != DF_OK) return st;
  DF_CUDA(launch_barrier_selftest(net->d_eng, limit_ns, net->stream));
  st = fail_if_device_error(net);
  // leave the network usable: clear the status word and the barrier state
  DF_CUDA(cudaMemsetAsync(&net->d_eng->status, 0, 2 * sizeof(int32_t), net->stream));
  DF_CUDA(cudaMemsetAsync(&net->d_eng->bar_arrive, 0, sizeof(unsigned long long) + sizeof(unsigned int),
                          net->stream));
  DF_CUDA(cudaStreamSynchronize(net->stream));
  return st;
}

df_status df_dpd_set_tile(df_net* net, int32_t actor, uint32_t tile, uint32_t threads) {
  if (!net || actor < 0 || actor >= (int)net->actors.size()) return DF_EINVAL;
  if (net->actors[actor].kind != DF_DPD && net->actors[actor].kind != DF_DPD_FIR) return DF_EINVAL;
  if (tile || threads) {
    if (threads != 32 && threads != 64 && threads != 128 && threads != 256) return DF_EINVAL;
    const uint32_t R = tile / threads;
    if (tile != R * threads || (R != 8 && R != 16)) return DF_EINVAL;
  }
  net->actors[actor].tile = tile;
  net->actors[actor].threads = threads;
  for (auto& kv : net->graphs) cudaGraphExecDestroy(kv.second);
  net->graphs.clear();
  return DF_OK;
}

df_status df_profile_enable(df_net* net, int32_t on) {
  if (!net) return DF_EINVAL;
  DeviceGuard g(net->device);
  const df_status st = prof_collect(net);
  if (st != DF_OK) return st;
  net->prof = on != 0;
  for (int i = 0; i < 4; ++i) {
    net->prof_ms[i] = 0;
    net->prof_n[i] = 0;
  }
  return DF_OK;
}

df_status df_profile_get(df_net* net, int32_t what, double* total_ms, uint64_t* launches) {
  if (!net || what < 0 || what > 3) return DF_EINVAL;
  DeviceGuard g(net->device);
  const df_status st = prof_collect(net);
  if (st != DF_OK) return st;
  if (total_ms) *total_ms = net->prof_ms[what];
  if (launches) *launches = net->prof_n[what];
  return DF_OK;
}

df_status df_autotune(df_net* net, uint64_t* n_firings) {
  if (!net) return DF_EINVAL;
  if (!net->finalized) return DF_ESTATE;
  DeviceGuard g(net->device);
  cudaStream_t s = net->stream;
  static const uint32_t kCand[][2] = {{256, 32},   {512, 32},   {512, 64},  {1024, 128}, {2048, 256},
                                      {1024, 64},  {2048, 128}, {4096, 256}};
  uint64_t before = 0;
  DF_CUDA(cudaStreamSynchronize(s));
  DF_CUDA(cudaMemcpy(&before, &net->d_eng->fired_total, 8, cudaMemcpyDeviceToHost));
  cudaEvent_t e0, e1;
  DF_CUDA(cudaEventCreate(&e0));
  DF_CUDA(cudaEventCreate(&e1));
  df_status st = DF_OK;
  for (const Op& op : net->program) {
    if (op.kind == kOpCopy) {
      DF_CUDA(launch_copy(op.copy, net->n_sm, s));
    } else if (op.kind == kOpMd) {
      DF_CUDA(launch_md_step(op.md, &op.md_tma, net->n_sm, s));
    } else if (op.kind == kOpDyn) {
      DF_CUDA(launch_dyn(op.dyn, net->n_sm, s));
    } else if (op.kind == kOpImg) {
      DF_CUDA(launch_img(op.img, net->n_sm, s));
    } else {
      // one plan, then the (idempotent) body once per candidate; keep the fastest
      DF_CUDA(launch_dpd_plan(op.dpd_dev, op.dpd_n, s));
      float best = 1e30f;
      uint32_t bt = 0, bth = 0;
      for (const auto& c : kCand) {
        for (int rep = 0; rep < 2; ++rep) {
          DF_CUDA(cudaEventRecord(e0, s));
          const cudaError_t le =
              launch_dpd_body(op.dpd_dev, op.dpd_order, op.dpd_n, c[0], c[1], op.max_mt, net->n_sm, s);
          if (le != cudaSuccess) {
            cudaGetLastError();            // configuration does not fit: skip it
            break;
          }
          DF_CUDA(cudaEventRecord(e1, s));
          DF_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          DF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (rep == 1 && ms < best) {     // second run: warm caches and clocks
            best = ms;
            bt = c[0];
            bth = c[1];
          }
        }
      }
      if (bt) {
        DF_CUDA(launch_dpd_body(op.dpd_dev, op.dpd_order, op.dpd_n, bt, bth, op.max_mt, net->n_sm, s));
        net->actors[op.dpd_first_actor].tile = bt;
        net->actors[op.dpd_first_actor].threads = bth;
      } else {
        st = DF_ENOTSUP;
      }
    }
    for (const SpillArgs& sp : op.spills) DF_CUDA(launch_spill(sp, s));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& kv : net->graphs) cudaGraphExecDestroy(kv.second);
  net->graphs.clear();
  if (st != DF_OK) return st;
  st = fail_if_device_error(net);
  if (st != DF_OK) return st;
  if (n_firings) {
    uint64_t after = 0;
    DF_CUDA(cudaMemcpy(&after, &net->d_eng->fired_total, 8, cudaMemcpyDeviceToHost));
    *n_firings = after - before;
  }
  return DF_OK;
}

df_status df_dpd_get_tile(df_net* net, int32_t actor, uint32_t* tile, uint32_t* threads) {
  if (!net || actor < 0 || actor >= (int)net->actors.size()) return DF_EINVAL;
  if (tile) *tile = net->actors[actor].tile;
  if (threads) *threads = net->actors[actor].threads;
  return DF_OK;
}

df_status df_dpd_forward(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                         const int32_t* orders, void* y, void* cuda_stream) {
  if ((!x || !y) && n) return DF_EINVAL;
  if (!h || !orders || K < 1 || K > DF_MAX_BRANCHES || M < 1 || M > DF_MAX_TAPS) return DF_EINVAL;
  for (int k = 0; k < K; ++k)
    if (orders[k] < 1 || orders[k] % 2 == 0 || orders[k] > 63) return DF_EINVAL;
  return cuda_status(dpd_forward_stateless(static_cast<const float2*>(x), n,
                                           static_cast<const float2*>(h), K, M, orders,
                                           static_cast<float2*>(y),
                                           static_cast<cudaStream_t>(cuda_stream)));
}

static df_status check_dpd_args(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                                const int32_t* orders, const void* grad_y, const void* grad_h) {
  if (((!x || !grad_y) && n) || !grad_h) return DF_EINVAL;
  if (!h || !orders || K < 1 || K > DF_MAX_BRANCHES || M < 1 || M > DF_MAX_TAPS) return DF_EINVAL;
  for (int k = 0; k < K; ++k)
    if (orders[k] < 1 || orders[k] % 2 == 0 || orders[k] > 63) return DF_EINVAL;
  return DF_OK;
}

df_status df_dpd_backward(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                          const int32_t* orders, const void* grad_y, void* grad_x, void* grad_h,
                          void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, grad_y, grad_h);
  if (st != DF_OK) return st;
  int dev = 0;
  DF_CUDA(cudaGetDevice(&dev));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t need = std::max<size_t>(1, dpd_backward_scratch_elems(n, K, M)) * sizeof(float2);
  // the lock is held until the kernels are enqueued
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  Scratch& sc = g_scratch[{dev, reinterpret_cast<uintptr_t>(s)}];
  if (sc.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DF_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return DF_ESTATE;   // no allocation inside a capture
    const size_t grow = std::max(need, 2 * sc.bytes);
    void* p = nullptr;
    if (cudaMalloc(&p, grow) != cudaSuccess) {
      cudaGetLastError();
      return DF_ENOMEM;
    }
    if (sc.ptr) g_scratch_retired.push_back(sc.ptr);
    sc.ptr = p;
    sc.bytes = grow;
  }
  return cuda_status(dpd_backward_stateless(
      static_cast<const float2*>(x), n, static_cast<const float2*>(h), K, M, orders,
      static_cast<const float2*>(grad_y), static_cast<float2*>(grad_x),
      static_cast<float2*>(grad_h), static_cast<float2*>(sc.ptr), sc.bytes / sizeof(float2), s));
}

df_status df_dpd_forward_f64(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                             const int32_t* orders, void* y, void* cuda_stream) {
  if ((!x || !y) && n) return DF_EINVAL;
  df_status st = check_dpd_args(x, n, h, K, M, orders, x, h);
  if (st != DF_OK) return st;
  return cuda_status(dpd_forward_stateless_f64(static_cast<const double2*>(x), n, static_cast<const double2*>(h),
                                               K, M, orders, static_cast<double2*>(y),
                                               static_cast<cudaStream_t>(cuda_stream)));
}

df_status df_dpd_backward_f64(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                              const int32_t* orders, const void* grad_y, void* grad_x, void* grad_h,
                              void* scratch, uint64_t scratch_elems, void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, grad_y, grad_h);
  if (st != DF_OK) return st;
  if (!scratch || scratch_elems < df_dpd_backward_scratch_elems(n, K, M)) return DF_EINVAL;
  return cuda_status(dpd_backward_stateless_f64(
      static_cast<const double2*>(x), n, static_cast<const double2*>(h), K, M, orders,
      static_cast<const double2*>(grad_y), static_cast<double2*>(grad_x), static_cast<double2*>(grad_h),
      static_cast<double2*>(scratch), scratch_elems, static_cast<cudaStream_t>(cuda_stream)));
}

uint64_t df_dpd_mse_partial_elems(uint64_t n) { return dpd_mse_partial_elems(n); }

df_status df_dpd_mse_forward(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                             const int32_t* orders, const void* target, void* resid, void* loss, void* partial,
                             uint64_t partial_elems, void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, target, resid);
  if (st != DF_OK) return st;
  if (!loss || !partial || partial_elems < dpd_mse_partial_elems(n)) return DF_EINVAL;
  return cuda_status(dpd_mse_forward(static_cast<const float2*>(x), n, static_cast<const float2*>(h), K, M, orders,
                                     static_cast<const float2*>(target), static_cast<float2*>(resid),
                                     static_cast<float*>(loss), static_cast<float*>(partial),
                                     static_cast<cudaStream_t>(cuda_stream)));
}

df_status df_dpd_mse_forward_f64(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                                 const int32_t* orders, const void* target, void* resid, void* loss,
                                 void* partial, uint64_t partial_elems, void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, target, resid);
  if (st != DF_OK) return st;
  if (!loss || !partial || partial_elems < dpd_mse_partial_elems(n)) return DF_EINVAL;
  return cuda_status(dpd_mse_forward_f64(static_cast<const double2*>(x), n, static_cast<const double2*>(h), K, M,
                                         orders, static_cast<const double2*>(target), static_cast<double2*>(resid),
                                         static_cast<double*>(loss), static_cast<double*>(partial),
                                         static_cast<cudaStream_t>(cuda_stream)));
}

df_status df_dpd_mse_backward(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                              const int32_t* orders, const void* resid, const void* grad_loss, void* grad_h,
                              void* scratch, uint64_t scratch_elems, void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, resid, grad_h);
  if (st != DF_OK) return st;
  if (!grad_loss || !scratch || scratch_elems < df_dpd_backward_scratch_elems(n, K, M)) return DF_EINVAL;
  return cuda_status(dpd_mse_backward(static_cast<const float2*>(x), n, static_cast<const float2*>(h), K, M, orders,
                                      static_cast<const float2*>(resid), static_cast<const float*>(grad_loss),
                                      static_cast<float2*>(grad_h), static_cast<float2*>(scratch), scratch_elems,
                                      static_cast<cudaStream_t>(cuda_stream)));
}

df_status df_dpd_mse_backward_f64(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                                  const int32_t* orders, const void* resid, const void* grad_loss, void* grad_h,
                                  void* scratch, uint64_t scratch_elems, void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, resid, grad_h);
  if (st != DF_OK) return st;
  if (!grad_loss || !scratch || scratch_elems < df_dpd_backward_scratch_elems(n, K, M)) return DF_EINVAL;
  return cuda_status(dpd_mse_backward_f64(static_cast<const double2*>(x), n, static_cast<const double2*>(h), K, M,
                                          orders, static_cast<const double2*>(resid),
                                          static_cast<const double*>(grad_loss), static_cast<double2*>(grad_h),
                                          static_cast<double2*>(scratch), scratch_elems,
                                          static_cast<cudaStream_t>(cuda_stream)));
}

uint64_t df_dpd_backward_scratch_elems(uint64_t n, int32_t K, int32_t M) {
  if (K < 1 || K > DF_MAX_BRANCHES || M < 1 || M > DF_MAX_TAPS) return 0;
  return std::max<uint64_t>(1, dpd_backward_scratch_elems(n, K, M));
}

df_status df_dpd_backward_scratch(const void* x, uint64_t n, const void* h, int32_t K, int32_t M,
                                  const int32_t* orders, const void* grad_y, void* grad_x,
                                  void* grad_h, void* scratch, uint64_t scratch_elems,
                                  void* cuda_stream) {
  df_status st = check_dpd_args(x, n, h, K, M, orders, grad_y, grad_h);
  if (st != DF_OK) return st;
  if (!scratch || scratch_elems < df_dpd_backward_scratch_elems(n, K, M)) return DF_EINVAL;
  return cuda_status(dpd_backward_stateless(
      static_cast<const float2*>(x), n, static_cast<const float2*>(h), K, M, orders,
      static_cast<const float2*>(grad_y), static_cast<float2*>(grad_x),
      static_cast<float2*>(grad_h), static_cast<float2*>(scratch), scratch_elems,
      static_cast<cudaStream_t>(cuda_stream)));
}

}  // extern "C"
