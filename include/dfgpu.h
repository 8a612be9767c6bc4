/*
 * dfgpu.h -- C ABI of the dynamic-data-rate dataflow engine for one B300 (sm_103a).
 *
 * The engine executes actor networks in the sense of Boutellier & Hautala,
 * "Executing Dynamic Data Rate Actor Networks on OpenCL Platforms" (SiPS 2016):
 *
 *   - a network is a set of actors joined by order-preserving FIFO channels
 *     (Sec. 2.2); a channel joins one output port to one input port (Sec. 3.2);
 *   - every channel has a token rate r > 0 adopted by both end ports (Sec. 2.2);
 *   - a dynamic actor owns one control input port of rate 1; per firing it
 *     consumes one control token, which fixes each regular port's rate to 0 or
 *     r for that firing (Sec. 2.2, the control function of Sec. 3.1);
 *   - channels not attached to a control port may hold initial (delay) tokens
 *     (Sec. 2.2; more than one is the generalisation mentioned in Sec. 3.2).
 *
 * Execution model.  df_run(n) performs n steps on the device.  A step visits
 * the actors in the order they were added and fires each one as many times as
 * it is enabled (the longest prefix of its pending firings whose cumulative
 * consumption fits the tokens present and whose cumulative production fits
 * the free space).  All rate decisions, scans, gathers and scatters happen in
 * CUDA kernels; the host is not involved between firings.  The resulting
 * channel contents equal those of a sequential interpreter that fires one
 * actor at a time (Kahn determinism).
 *
 * Memory.  A network owns every device buffer it allocates (channel rings,
 * counters, per-actor state); df_net_destroy frees them.  Channels are ring
 * buffers of `capacity` tokens of `token_bytes` bytes, token i of the stream
 * living in slot i mod capacity (or laid out as in Sec. 3.2, Eq. 1 and Fig. 2,
 * see DF_CAPACITY_EQ1).  Push and pop copy (the caller keeps its buffers).  All device work of a network is ordered on its stream.
 *
 * Errors.  Every call returns a df_status; DF_OK (0) on success, a negative
 * code otherwise.  Out-parameters are written only on success.  No call aborts
 * the process.  Device-side waits are bounded: a wait that runs out reports
 * DF_ETIMEOUT through the network's status word instead of hanging.
 *
 * Thread safety: a network must not be used from two host threads at once.
 */
#ifndef DFGPU_H
#define DFGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t df_status;
enum {
    DF_OK = 0,
    DF_EINVAL = -1,      /* invalid argument or network (validation failure) */
    DF_ENOMEM = -2,      /* device or host allocation failed */
    DF_EFULL = -3,       /* push does not fit the free space of every output channel */
    DF_EEMPTY = -4,      /* nothing to pop where tokens were required */
    DF_ESTATE = -5,      /* call not allowed in the network's current state */
    DF_EDEADLOCK = -6,   /* run(-1) stopped without reaching quiescence within its step limit */
    DF_ETIMEOUT = -7,    /* a bounded device-side wait ran out */
    DF_ECUDA = -8,       /* a CUDA runtime call failed */
    DF_ENOTSUP = -9      /* configuration outside what the kernels implement */
};

/* Actor kinds (df_actor_add).  Port numbering is per kind; for every dynamic
 * kind input port 0 is the control port (rate 1, u32 token = bit mask). */
enum {
    DF_SOURCE = 1,    /* host push endpoint; out ports 0..n-1 each receive every pushed token */
    DF_SINK = 2,      /* host pop endpoint; in port 0 */
    DF_COPY = 3,      /* static: in 0 -> every out port; bytes per firing equal on all ports */
    DF_DPD = 4,       /* dynamic fused predistorter (Sec. 4.2): in 0 ctrl, in 1 data, out 0;
                         params df_dpd_params; all ports rate 1; token = block_len complex64 */
    DF_DPD_POLY = 5,  /* dynamic (Sec. 4.2 "P"): in 0 ctrl, in 1 data -> out k = branch k signal */
    DF_DPD_FIR = 6,   /* static FIR of one branch: in 0 -> out 0, rate 1 */
    DF_DPD_ADD = 7,   /* dynamic (Sec. 4.2 "A"): in 0 ctrl, in k+1 branch k -> out 0 */
    DF_MD = 8,        /* fused motion detector: in 0 current frame, in 1 previous frame;
                         out 0 tile records (variable rate, r_max = tiles per frame),
                         out 1 per-frame record count (u32); params df_md_params */
    /* The paper's own motion pipeline (Sec. 4.1): static image actors on
     * u8 frames (token_bytes = width*height), params df_img_params, every
     * port of an actor at the same rate r (r frames per firing). */
    DF_GAUSS5 = 9,    /* "Gauss": in 0 -> every out port: 5x5 binomial filter (weights
                         (1,4,6,4,1) x (1,4,6,4,1) / 256, rounded half up, columns clamped
                         at the edges) of rows 2..height-3; rows 0, 1, height-2, height-1
                         copied unfiltered */
    DF_THRES = 10,    /* "Thres": in 0 current frame, in 1 previous frame -> out 0:
                         255 where |cur - prev| > threshold, else 0 */
    DF_MED5 = 11      /* "Med": in 0 -> every out port: median of each pixel and its 4
                         nearest neighbours; the outermost rows and columns copied */
};

#define DF_MAX_BRANCHES 16
#define DF_MAX_TAPS 32

/* Predistorter parameters (DF_DPD, DF_DPD_POLY, DF_DPD_FIR, DF_DPD_ADD).
 * Branch k computes z_k = |x|^(orders[k]-1) x (orders odd, >= 1), filters it
 * with the M-tap complex FIR h[k*M .. k*M+M-1], and the active branches are
 * summed in ascending k.  A branch's FIR sees only the blocks in which the
 * branch was active (its input stream is the compaction of those blocks).
 * h is complex64 interleaved (re, im), host memory, copied at df_actor_add.
 * DF_DPD_POLY uses K/orders; DF_DPD_FIR uses M and h of branch `branch`;
 * DF_DPD_ADD uses K and block_len. */
typedef struct {
    int32_t K;                          /* branches, 1..DF_MAX_BRANCHES */
    int32_t M;                          /* taps, 1..DF_MAX_TAPS */
    int32_t orders[DF_MAX_BRANCHES];    /* odd polynomial order per branch */
    uint32_t block_len;                 /* samples per token (complex64) */
    int32_t branch;                     /* DF_DPD_FIR only: which row of h */
    const float *h;                     /* K*M complex64 (2*K*M floats), host */
} df_dpd_params;

/* Motion-detector parameters (DF_MD).  Frames are height x width uint8,
 * row-major (token_bytes = width*height).  A pixel is moving iff
 * |cur - prev| > threshold; the mask is opened by a 3x3 erosion (pixels
 * outside the frame count as set) then a 3x3 dilation (outside counts as
 * clear); for every 16x16 tile (raster order, partial last tile row allowed)
 * with count > 0 one 8-byte record {u16 x, u16 y, u32 count} is emitted, x/y
 * being the tile's top-left pixel.  width must be a multiple of 32 and tile
 * 16: other valid sizes return DF_ENOTSUP from df_actor_add. */
typedef struct {
    int32_t width;
    int32_t height;
    int32_t threshold;                  /* 25 in the benchmark */
    int32_t tile;                       /* must be 16 */
} df_md_params;

/* Image-actor parameters (DF_GAUSS5, DF_THRES, DF_MED5).  width must be a
 * multiple of 16 and at most 2048 (other widths return DF_ENOTSUP from
 * df_actor_add); threshold (DF_THRES) in 0..255. */
typedef struct {
    int32_t width;
    int32_t height;
    int32_t threshold;                  /* DF_THRES only; 20 in the paper-pipeline workload */
} df_img_params;

typedef struct df_net df_net;

/* Create an empty network on `device`.  `cuda_stream` is a cudaStream_t the
 * network will use for all its work (NULL: the network creates and owns a
 * non-blocking stream).  *out receives the handle.
 * Defined by: Sec. 2.2 (a network is a set of actors and a set of FIFO
 * channels) and Sec. 3.4 (the application declares its network through the
 * framework's C library). */
df_status df_net_create(df_net **out, int device, void *cuda_stream);

/* Free every resource of the network (NULL-safe).  Waits for its stream.
 * Defined by: Sec. 3.3 (the framework's threads and buffers live from the
 * start of the application to its end). */
void df_net_destroy(df_net *net);

/* Add an actor of `kind` with kind-specific `params` (copied).  Returns its
 * id in *out_id; ids are dense and give the step order (Sec. 3.3 leaves the
 * schedule to the OS; this engine fixes it to insertion order).
 * Defined by: Sec. 2.2 (static actors, dynamic actors with a control port)
 * and Sec. 3.1 (an actor's init, fire and control functions: init is this
 * call, fire and control run on the device); the actor kinds are those of
 * Sec. 4.1 and Sec. 4.2. */
df_status df_actor_add(df_net *net, int32_t kind, const void *params, size_t params_bytes,
                       int32_t *out_id);

/* Connect output port src_port of src_actor to input port dst_port of
 * dst_actor by a FIFO of `capacity_tokens` tokens of `token_bytes` bytes with
 * token rate `rate` (Sec. 2.2).  `initial_tokens` delay tokens are present
 * before any firing; their contents come from `initial_data` (host,
 * initial_tokens*token_bytes bytes) or are zero when it is NULL.  Control
 * channels need rate 1 and no initial tokens.  capacity must be >= initial +
 * rate.  Self-loops (src_actor == dst_actor) are rejected.
 *
 * capacity_tokens == DF_CAPACITY_EQ1 selects the paper's own channel layout
 * (Sec. 3.2): the buffer size is not chosen by the caller but set by Eq. 1,
 * 2r slots (a double buffer) without a delay token and 3r+1 slots with one,
 * and a channel with a delay token follows the access pattern of Fig. 2: the
 * delay token sits in slot 0, write k fills slots 1+(kr mod 3r) .. +r-1, read
 * k takes slots (kr mod 3r) .. +r-1, and the write that fills slot 3r is
 * followed by a copy of slot 3r into slot 0.  Every window of r tokens is then
 * one contiguous run of slots.  Such a channel holds at most 2r (no delay) or
 * 3r (delay) unread tokens: one more window of r would overwrite a token
 * not yet read.  Pushes into it write whole windows (n_tokens a multiple of
 * r, else DF_EINVAL).  initial_tokens must be 0 or 1 (the paper gives the pattern
 * for one delay token) and the writer must be a host source or an actor of a
 * fixed token rate per firing (not the output of DF_MD); else DF_EINVAL.
 * Defined by: Sec. 2.2 (order-preserving FIFO between one output and one input
 * port, token rate, initial tokens), Sec. 3.2 (capacity, Eq. 1, Fig. 2). */
#define DF_CAPACITY_EQ1 0u
df_status df_channel_connect(df_net *net, int32_t src_actor, int32_t src_port,
                             int32_t dst_actor, int32_t dst_port, uint32_t token_bytes,
                             uint32_t rate, uint32_t capacity_tokens, uint32_t initial_tokens,
                             const void *initial_data, int32_t *out_ch);

/* Validate (ports connected exactly once and numbered densely, rates and token
 * sizes consistent with each actor kind), plan and allocate device memory.
 * The network is frozen afterwards.
 * Defined by: Sec. 2.2 (control channels have rate 1 and no initial tokens;
 * one channel per port) and Sec. 3.2 (every buffer is allocated before the
 * actors start, at its fixed size). */
df_status df_net_finalize(df_net *net);

/* Copy n_tokens tokens (n_tokens*token_bytes bytes at `src`, host or device
 * memory) into every output channel of source actor `src_actor`.
 * All-or-nothing: DF_EFULL when any channel lacks space (nothing written).
 * Defined by: Sec. 3.3 and Sec. 4 (host-side source actors feed the network:
 * video frames read by the CPU, predistorter input blocks); a write that lacks
 * space is refused here instead of blocking as in Sec. 3.3. */
df_status df_push(df_net *net, int32_t src_actor, const void *src, uint64_t n_tokens,
                  uint64_t *n_pushed);

/* Run n_steps steps (n_steps < 0: until a step fires nothing, at most 2^20
 * steps, else DF_EDEADLOCK).  Blocks until the device work is done, then
 * reports the device status word and, if non-NULL, the number of firings.
 * Defined by: Sec. 2.2 (the firing rule of a dynamic actor: read one control
 * token, fix the port rates, consume, compute, produce), with Sec. 3.3's free-
 * running actor threads read as steps: each step fires every actor, in
 * insertion order, while it is enabled. */
df_status df_run(df_net *net, int64_t n_steps, uint64_t *n_firings);

/* Run flags for df_run_ex. */
enum {
    DF_RUN_ASYNC = 1,        /* enqueue only (n_steps >= 0); no host sync, no firing count */
    DF_RUN_GRAPH = 2,        /* replay a CUDA graph of n_steps steps (captured once per n); with
                                DF_RUN_PERSISTENT the graph holds the one persistent launch */
    DF_RUN_PERSISTENT = 4,   /* one cooperative persistent kernel runs all steps (for n_steps < 0
                                also the quiescence check); phases are separated by a grid
                                barrier bounded by the wait limit (df_set_wait_limit) */
    DF_RUN_NO_BATCH = 8      /* one launch per predistorter actor instead of one per group */
};
/* df_run with flags.  Defined by: Sec. 2.2 as df_run; the flags choose how the
 * steps are launched (Sec. 3.3's contrast: no host round trip per firing). */
df_status df_run_ex(df_net *net, int64_t n_steps, uint32_t flags, uint64_t *n_firings);

/* Wait for the network's stream and return the device status word (DF_OK or
 * the first device-side error) and the total number of firings so far.
 * Defined by: Sec. 3.3 (the host learns of the GPU actors' progress); the
 * firing count is the Sec. 2.2 firing counted on the device. */
df_status df_sync(df_net *net, uint64_t *total_firings);

/* Copy up to max_tokens tokens from the input channel of sink `sink_actor`
 * into `dst` (host or device memory).  Blocks until the copy is done.
 * Defined by: Sec. 3.3 and Sec. 4 (host-side sink actors consume the
 * network's output). */
df_status df_pop(df_net *net, int32_t sink_actor, void *dst, uint64_t max_tokens,
                 uint64_t *n_popped);

/* Concurrent host I/O: the paper's host actors (Sec. 3.3, 4) run in threads of
 * their own beside the GPU actors.  With DF_IO_CONCURRENT a push (pop) runs on
 * a stream of its own, so that its copies overlap df_run's kernels and the
 * other direction's copies; without the flag these equal df_push / df_pop.
 * The free space (tokens present) is taken from a snapshot of the channel's
 * counters, which a concurrent consumer (producer) can only have increased,
 * so the call may see less than there is but never more.  The tokens are
 * copied before the counter moves, on the same stream.  At most one thread
 * may push to a given source and one pop from a given sink at a time; calls
 * with the flag may run concurrently with df_run, df_sync and each other
 * (different sources and sinks from different threads).  df_push/df_pop and
 * df_channel_counters stay on the network's stream and belong to the thread
 * that runs it.
 * Defined by: Sec. 3.3 (every actor a thread of its own, host and GPU actors
 * running concurrently) and Sec. 1 (concurrent CPU and GPU actors). */
enum { DF_IO_CONCURRENT = 1 };
df_status df_push_ex(df_net *net, int32_t src_actor, const void *src, uint64_t n_tokens,
                     uint32_t flags, uint64_t *n_pushed);
df_status df_pop_ex(df_net *net, int32_t sink_actor, void *dst, uint64_t max_tokens,
                    uint32_t flags, uint64_t *n_popped);

/* Native runner of the paper's host actors (Sec. 3.3: every actor an OS
 * thread, a read that lacks tokens blocks until they arrive).  One host
 * thread per feed pushes its tokens in batches of `batch` (a batch that does
 * not fit is retried once a step or a pop has freed space), one thread per
 * drain pops up to `batch` tokens at a time into consecutive places of
 * `data`, and the calling thread runs the GPU actors one step at a time
 * (df_run_ex with run_flags, which must not contain DF_RUN_ASYNC).  All I/O
 * uses DF_IO_CONCURRENT, so its copies overlap the steps.  The run ends when
 * every feed is pushed, a step fires nothing, every drained sink's channel is
 * empty and one more step fires nothing; drains[i].n_popped then holds the
 * tokens popped (a drain also stops when max_tokens are in).  When nothing
 * moves (no firing, push or pop) for idle_limit_ns (<= 0: 2 s) the run stops
 * with DF_EDEADLOCK, e.g. when an undrained sink is full.  Feed data may be
 * host (pinned for full speed) or device memory, as for df_push.
 * Defined by: Sec. 3.3 (one OS thread per actor, blocking FIFO reads and
 * writes) for the host actors; the GPU actors run as df_run. */
typedef struct {
    int32_t source;          /* DF_SOURCE actor */
    const void *data;        /* n_tokens tokens */
    uint64_t n_tokens;
    uint64_t batch;          /* tokens per push (a multiple of r for Eq. 1 channels) */
} df_feed;
typedef struct {
    int32_t sink;            /* DF_SINK actor */
    void *data;              /* room for max_tokens tokens */
    uint64_t max_tokens;
    uint64_t batch;          /* tokens per pop, at most */
    uint64_t n_popped;       /* out */
} df_drain;
df_status df_stream(df_net *net, const df_feed *feeds, int32_t n_feeds, df_drain *drains,
                    int32_t n_drains, uint32_t run_flags, int64_t idle_limit_ns, uint64_t *n_steps);

/* Counters of channel `ch`: tokens produced (excluding initial tokens),
 * consumed, and currently held.  produced + initial == consumed + occupancy.
 * Defined by: Sec. 2.2 (a FIFO channel delivers the tokens written to it, in
 * order, plus its initial tokens). */
df_status df_channel_counters(df_net *net, int32_t ch, uint64_t *produced, uint64_t *consumed,
                              uint64_t *occupancy);

/* Layout and size of channel `ch`: capacity = the most unread tokens it can
 * hold; slots = buffer slots allocated (capacity, or capacity + 1 for a
 * delay channel in the paper's layout); buffer_bytes = slots * token_bytes;
 * layout = DF_LAYOUT_RING or DF_LAYOUT_EQ1.  Valid before and after
 * finalize.  Defined by: Sec. 3.2 (Eq. 1) and Table 1 (buffer memory). */
enum { DF_LAYOUT_RING = 0, DF_LAYOUT_EQ1 = 1 };
typedef struct {
    uint64_t capacity;
    uint64_t slots;
    uint64_t buffer_bytes;
    uint32_t token_bytes;
    uint32_t rate;
    uint32_t initial_tokens;
    int32_t layout;
} df_channel_info_t;
df_status df_channel_info(df_net *net, int32_t ch, df_channel_info_t *out);

/* Copy n_slots raw buffer slots of channel `ch`, starting at slot first_slot,
 * to `dst` (host), whatever tokens they hold: the physical layout (ring or
 * Fig. 2) made visible for inspection.  Runs on the network's stream and
 * blocks; DF_EINVAL when the range exceeds the slots of the channel.
 * Defined by: Sec. 3.2 and Fig. 2 (the slots of the double and triple buffer). */
df_status df_channel_peek_slots(df_net *net, int32_t ch, uint64_t first_slot, uint64_t n_slots,
                                void *dst);

/* Tile configuration of the predistorter kernel for one actor (0 = default):
 * samples per tile and threads per CTA (32, 64, 128 or 256; 8 or 16 samples
 * per thread, else DF_EINVAL).  The autotuner sets these.
 * The paper has no counterpart: a launch parameter of this engine's kernel
 * for the Sec. 4.2 predistorter. */
df_status df_dpd_set_tile(df_net *net, int32_t actor, uint32_t tile, uint32_t threads);

/* Time every supported tile configuration on the network's current pending
 * predistorter work (the firings a step would take now) and keep the fastest
 * for every DF_DPD actor / group.  Runs one step; returns its firings.
 * The paper has no counterpart (the tile autotuner of this engine). */
df_status df_autotune(df_net *net, uint64_t *n_firings);

/* The tile configuration an actor (the first actor of a batched group) uses;
 * 0/0 = the default.  The paper has no counterpart. */
df_status df_dpd_get_tile(df_net *net, int32_t actor, uint32_t *tile, uint32_t *threads);

/* Kernel timing.  While enabled, every non-graph step records CUDA events on
 * the network's stream around the kernels named below; df_profile_get waits
 * for the stream and returns their summed device time (ms) and launch count
 * since the last enable.  Graph replays (DF_RUN_GRAPH) are not timed.
 * The paper has no counterpart (measurement of this engine's kernels). */
enum {
    DF_PROF_STEP = 0,        /* one whole step (every launch of the step) */
    DF_PROF_DPD_BODY = 1,    /* predistorter body launches */
    DF_PROF_MD_MAIN = 2,     /* motion-detector streaming kernel */
    DF_PROF_COPY_BODY = 3    /* copy-actor body launches */
};
df_status df_profile_enable(df_net *net, int32_t on);
df_status df_profile_get(df_net *net, int32_t what, double *total_ms, uint64_t *launches);

/* Upper bound, in nanoseconds, of every device-side wait of the network (the
 * persistent kernel's grid barrier, the motion kernel's and the image actors'
 * staging waits); default one second.  A wait that runs out records
 * DF_ETIMEOUT in the status word and the kernel returns; the status word stays
 * set (df_run returns it, and persistent launches do nothing while it is set).
 * The paper has no counterpart (its actors block on mutexes, Sec. 3.3). */
df_status df_set_wait_limit(df_net *net, int64_t limit_ns);

/* Self-test of the bounded waits: runs a grid barrier that waits for one more
 * CTA than it has, so it can only end by its limit.  Returns the status word
 * that run left (DF_ETIMEOUT when the bound works), then clears it so the
 * network stays usable.  The paper has no counterpart. */
df_status df_selftest_wait_timeout(df_net *net, int64_t limit_ns);

/* Text for a status code (static storage).  The paper has no counterpart. */
const char *df_status_str(df_status s);

/* The failing CUDA call and its error string behind the calling thread's most
 * recent DF_ECUDA (empty if none); valid until the thread's next failure.
 * The paper has no counterpart. */
const char *df_last_error(void);

/* ---------------------------------------------------------------------------
 * Stateless predistorter operators (device pointers, caller's stream).
 * One contiguous signal of n samples, every branch active, zero history:
 *   y[t] = sum_k sum_{m<M} h[k,m] z_k[t-m],  z_k = |x|^(orders[k]-1) x,  z_k[<0] = 0.
 * x, y: n complex64; h: K*M complex64 (device); orders: host array of K ints.
 * ------------------------------------------------------------------------- */
/* Defined by: Sec. 4.2 (the predistorter: a Poly actor feeding parallel
 * FIR filters whose outputs an Adder sums), with every branch active on one
 * signal.  The paper does not print the branch function; it is read as the
 * memory-polynomial branch z_k above, with odd orders.  This is the form the
 * differentiable fit drives (indirect learning of the taps). */
df_status df_dpd_forward(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                         const int32_t *orders, void *y, void *cuda_stream);

/* Adjoint of df_dpd_forward for a real loss L.  grad_y, grad_x and grad_h use
 * the convention dL/dRe + i dL/dIm (PyTorch's for complex tensors):
 *   grad_h[k,m] = sum_t grad_y[t] conj(z_k[t-m])
 *   gz_k[j]     = sum_m conj(h[k,m]) grad_y[j+m]
 *   grad_x[j]   = sum_k (q_k+1) u^q_k gz_k[j] + q_k u^(q_k-1) x^2 conj(gz_k[j]),
 *                 u = |x[j]|^2, q_k = (orders[k]-1)/2.
 * grad_x may be NULL.  The z_k are recomputed from x, not stored.  grad_h is
 * reduced deterministically (fixed-order two-level sum).
 * Scratch: the tap-gradient partial sums live in a buffer the library
 * allocates per (device, stream) and grows on demand; a buffer is never freed
 * while the process runs (a grown one is retired, not released), so CUDA
 * graphs that captured an earlier call stay valid.  Calls on the same stream
 * are ordered by that stream; calls on different streams use different
 * buffers.  A call that would have to grow the buffer while its stream is
 * being captured returns DF_ESTATE (make one call of that size or larger
 * before capturing).  A graph captured from a call uses the buffer of the
 * stream it was captured on: replay it on that stream, or make sure no call
 * on that stream overlaps the replay.
 * Defined by: the adjoint of the Sec. 4.2 predistorter (df_dpd_forward); the
 * paper has no gradient, it is what fits the taps. */
df_status df_dpd_backward(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                          const int32_t *orders, const void *grad_y, void *grad_x, void *grad_h,
                          void *cuda_stream);

/* Scratch of the adjoint for callers that provide it: the number of complex64
 * elements df_dpd_backward_scratch needs for n samples, K branches and M taps
 * (ceil(n/1024) * K * MT, at least 1; MT = M rounded up to 4, 8, M for 9..16,
 * or 32); 0 for K or M out of range.
 * Defined by: the adjoint of the Sec. 4.2 predistorter, as df_dpd_backward;
 * the scratch itself has no counterpart in the paper. */
uint64_t df_dpd_backward_scratch_elems(uint64_t n, int32_t K, int32_t M);

/* df_dpd_backward with the tap-gradient partial sums in `scratch` (device
 * memory of at least df_dpd_backward_scratch_elems(n, K, M) complex64
 * elements, owned by the caller, else DF_EINVAL).  The call allocates
 * nothing, so it may be captured in a CUDA graph when the caller's allocator
 * is graph-aware (the torch binding passes a torch tensor).  Calls that
 * overlap on the GPU need different scratch buffers.
 * Defined by: the adjoint of the Sec. 4.2 predistorter (df_dpd_forward). */
df_status df_dpd_backward_scratch(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                                  const int32_t *orders, const void *grad_y, void *grad_x,
                                  void *grad_h, void *scratch, uint64_t scratch_elems,
                                  void *cuda_stream);

/* df_dpd_forward and df_dpd_backward_scratch in float64 arithmetic on
 * complex128 data (x, h, y, grad_y, grad_x, grad_h and the scratch, whose
 * element count is df_dpd_backward_scratch_elems(n, K, M) complex128 values).
 * They exist so that the hand-written adjoint can be checked against finite
 * differences at full precision (torch.autograd.gradcheck); FP64 throughput
 * on this GPU is a small fraction of FP32.
 * Defined by: the Sec. 4.2 predistorter and its adjoint, as the float32 forms. */
df_status df_dpd_forward_f64(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                             const int32_t *orders, void *y, void *cuda_stream);
df_status df_dpd_backward_f64(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                              const int32_t *orders, const void *grad_y, void *grad_x, void *grad_h,
                              void *scratch, uint64_t scratch_elems, void *cuda_stream);

/* The loss of the differentiable fit in the same kernels: resid = P_h(x) -
 * target (complex64, n values, P_h as df_dpd_forward), *loss = mean |resid|^2
 * (one float32 on the device), the tile sums of |resid|^2 added in a fixed
 * order through `partial` (device memory of at least
 * df_dpd_mse_partial_elems(n) float32, owned by the caller).  DF_EINVAL on a
 * missing pointer or a short `partial`.
 * Defined by: the indirect-learning fit of the Sec. 4.2 predistorter (the
 * paper has no loss; it is what fits the taps). */
uint64_t df_dpd_mse_partial_elems(uint64_t n);
df_status df_dpd_mse_forward(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                             const int32_t *orders, const void *target, void *resid, void *loss,
                             void *partial, uint64_t partial_elems, void *cuda_stream);
/* Gradient of that loss with respect to the taps: grad_h as df_dpd_backward
 * with grad_y = resid * (2 g / n), g = *grad_loss (one float32 on the device,
 * dL'/dloss of the caller's objective), without materialising grad_y; scratch
 * as df_dpd_backward_scratch.
 * Defined by: the indirect-learning fit of the Sec. 4.2 predistorter, as
 * df_dpd_mse_forward. */
df_status df_dpd_mse_backward(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                              const int32_t *orders, const void *resid, const void *grad_loss, void *grad_h,
                              void *scratch, uint64_t scratch_elems, void *cuda_stream);
/* df_dpd_mse_forward / df_dpd_mse_backward in float64 arithmetic on
 * complex128 data (loss, partial and grad_loss float64), for the
 * finite-difference check.
 * Defined by: the indirect-learning fit of the Sec. 4.2 predistorter, as
 * df_dpd_mse_forward. */
df_status df_dpd_mse_forward_f64(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                                 const int32_t *orders, const void *target, void *resid, void *loss,
                                 void *partial, uint64_t partial_elems, void *cuda_stream);
df_status df_dpd_mse_backward_f64(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                                  const int32_t *orders, const void *resid, const void *grad_loss,
                                  void *grad_h, void *scratch, uint64_t scratch_elems, void *cuda_stream);

/* Same computation and results as df_dpd_backward, but it allocates nothing.
 * (The paper has no counterpart; this exists for callers that may not
 * allocate device memory, e.g. a real-time adaptation loop where cudaMalloc
 * could synchronise the device and block, or a runtime with a fixed device
 * memory budget.)  The tap-gradient partial sums live in a fixed array inside
 * the library image: 131072 complex values (1 MiB) that every GPU loading the
 * library keeps until the process exits.  A call needs ceil(n/1024) * K * MT
 * of them (MT = M rounded up to 4, 8, M for 9..16, or 32); larger calls
 * return DF_ENOTSUP and do nothing.  Every call looks up the array's device
 * address (cudaGetSymbolAddress) on the current device; the first lookup on a
 * device may load the library's device code, so make the first call on each
 * device before any stream capture.  All calls share the one
 * array, so calls whose kernels overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Each call rewrites
 * every partial sum it reads, so nothing is carried over between calls. */
df_status df_dpd_backward_noalloc(const void *x, uint64_t n, const void *h, int32_t K, int32_t M,
                                  const int32_t *orders, const void *grad_y, void *grad_x,
                                  void *grad_h, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DFGPU_H */
