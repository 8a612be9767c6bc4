#!/usr/bin/env python3
"""Throughput benchmark of the dataflow engine on one B300 (and N ranks, weak scaling).

Headline workload: the motion-detection network on 300 synthetic 1920x1080
uint8 frames (source -> {current, previous with one initial frame} -> fused
detector -> record / count sinks).  One step = one engine step that fires the
detector on every frame resident in its input channel, i.e. one pass of the
whole path over the batch.  Secondary workloads in the same JSON line: the
large predistorter (512 blocks x 2^20 complex64, up to 8 branches, 16 taps),
the tiny predistorter (64 x 4096, capacity 8) and the batched and
differentiable forms.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--quick] [--only LIST]

The GPU arm prints one JSON line with the device-timed value, the end-to-end
value through the C ABI from pinned host memory, the roofline of the dominant
kernel (timed with CUDA events on the engine's stream), the oracle timed on
the host as CPU baseline, and the SM clocks seen while it ran.  The reference
arm (``--impl reference``) times the CPU oracle on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "DPD Msamples/s & motion-detect frames/s on 1 B300; % of HBM roofline"
SECONDARY = ("dpd_large", "dpd_tiny", "dpd_batch", "dpd_fit", "md_paper")
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (Blackwell)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2032.0)),
                "source": "measured"}
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0, "source": "fallback"}


def fp32_peak(pk, torch):
    """FP32 FMA peak of GPU 0 in TFLOP/s: SMs (from the device) x 128 lanes x 2 flop
    x the maximum SM clock."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    return n_sm * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12, n_sm


def profiled_traffic(summary):
    """DRAM bytes per launch from a profiles/ summary, or None when the kernel
    sources have changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    try:
        h = hashlib.sha256()
        for f in fields["sources"].split():
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest()[:16] != fields["source_sha256"]:
            return None
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, OSError, ValueError):
        return None


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "util": float(parts[4]),
                             "hw": parts[6], "hwt": parts[7], "swt": parts[8], "pcap": parts[9]})
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in busy:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in busy),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "samples_busy": len(busy)}


# ----------------------------------------------------------- distributed ----
def dist_setup(args):
    from paper_1611_03226_b300 import ranks
    return ranks.world()


def max_over_ranks(x, ws):
    from paper_1611_03226_b300 import ranks
    return ranks.max_over_ranks(x) if ws > 1 else x


def barrier(ws):
    from paper_1611_03226_b300 import ranks
    if ws > 1:
        ranks.barrier()


# ------------------------------------------------------- CPU baselines ----
# The oracle as it stands, timed on the host's cores in three ways: the
# sequential sweep interpreter on one core; the paper's runner with one OS
# thread per actor (Sec. 3.3) on the literal network; and independent
# replicas of the sequential oracle over contiguous ranges of the workload in
# one spawned process per core (each replica's run timed inside it; the range
# time is the slowest replica).
def host_info():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count() or 1, "cpu_model": model}


_POOL = None


def oracle_pool():
    """Process pool of one worker per host core, started with spawn (never
    forked from a process that holds a CUDA context)."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        _POOL = mp.get_context("spawn").Pool(os.cpu_count() or 1)
    return _POOL


def _motion_range(args):
    """Oracle motion network over frames t0 .. t1-1 of the T-frame workload; the
    frame before t0 is the previous-frame channel's initial token."""
    t0, t1, T, H, W = args
    from oracle import nets as ON
    w = synth.motion(n_frames=T, height=H, width=W)
    prev = w.frame(t0 - 1) if t0 > 0 else None
    net, ids = ON.motion_fused(H, W, t1 - t0 + 1, prev_init=prev)
    net.push(ids["src"], [w.frame(t) for t in range(t0, t1)])
    start = time.perf_counter()
    n = net.run(-1)
    return time.perf_counter() - start, n


def _dpd_large_range(args):
    """Oracle fused predistorter over blocks b0 .. b1-1 of the large workload
    as an independent stream (zero history, no delay blocks)."""
    b0, b1 = args
    from oracle import nets as ON
    w = synth.dpd_large()
    net, ids = ON.dpd_fused(w.h, w.orders, w.block_len, 0, b1 - b0)
    net.push(ids["ctrl"], ON.as_tokens_ctrl(w.masks[b0:b1]))
    net.push(ids["data"], ON.as_tokens_blocks([w.block(b) for b in range(b0, b1)]))
    start = time.perf_counter()
    n = net.run(-1)
    return time.perf_counter() - start, n * w.block_len


def _dpd_batch_channel(c):
    """Oracle fused predistorter of channel c of the batched workload (16 blocks)."""
    from oracle import nets as ON
    w = synth.dpd_batch()
    nb, L = w.blocks_per_channel, int(w.lengths[c])
    net, ids = ON.dpd_fused(w.h[c], w.orders, L, 0, nb)
    net.push(ids["ctrl"], ON.as_tokens_ctrl([int(w.masks[c])] * nb))
    net.push(ids["data"], ON.as_tokens_blocks([w.block(c, b) for b in range(nb)]))
    start = time.perf_counter()
    net.run(-1)
    return time.perf_counter() - start, nb * L


def _md_paper_range(args):
    """The paper's pipeline (oracle network, rate 4) over frames t0 .. t1-1."""
    t0, t1, T, H, W, thr = args
    from oracle import motion_paper as MP
    from oracle import nets as ON
    w = synth.motion(n_frames=T, height=H, width=W)
    init = MP.gauss5(w.frame(t0 - 1)) if t0 > 0 else None
    net, ids = ON.motion_paper(H, W, t1 - t0 + 4, 4, thr, initial=init)
    net.push(ids["src"], [w.frame(t) for t in range(t0, t1)])
    start = time.perf_counter()
    net.run(-1)
    return time.perf_counter() - start, t1 - t0


def parallel_oracle(fn, parts):
    """Run fn over parts in the process pool; returns (slowest replica's run
    time, summed units, processes used)."""
    res = oracle_pool().map(fn, parts)
    return max(r[0] for r in res), sum(r[1] for r in res), len(parts)


def split(n, k):
    """k contiguous ranges covering 0 .. n-1."""
    b = [round(i * n / k) for i in range(k + 1)]
    return [(b[i], b[i + 1]) for i in range(k) if b[i + 1] > b[i]]


def threaded_motion(frames, H, W, n):
    """Thread-per-actor runner (Sec. 3.3) on the literal five-actor motion network."""
    from oracle import nets as ON
    net, ids = ON.motion_literal(H, W, n + 1)
    net.push(ids["src"], list(frames[:n]))
    start = time.perf_counter()
    fired = net.run_threaded()
    dt = time.perf_counter() - start
    return {"value": n / dt, "unit": "frames/s", "threads": 5, "firings": fired,
            "sample": f"first {n} frames; Diff, Thresh, Erode, Dilate and Tiles as one thread each"}


# ------------------------------------------------------------ workloads ----
def gen_parallel(fn, n, workers=16):
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, range(n)))


def flush_l2(buf):
    """Evict L2 before a timed step: write one buffer larger than L2 (256 MB),
    then read a second one, so that the step finds neither its inputs nor the
    flush's dirty lines in L2 (their write-back to DRAM would otherwise fall in
    the timed region and be charged to the kernel)."""
    buf[0].add_(1)
    buf[1].amax()


def motion_net(P, torch, T, H, W, thr=25):
    n_tiles = (-(-H // 16)) * (-(-W // 16))
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    src, md = net.add_source(), net.add_md(W, H, thr)
    rec, cnt = net.add_sink(), net.add_sink()
    net.connect(src, 0, md, 0, W * H, 1, T + 1)
    net.connect(src, 1, md, 1, W * H, 1, T + 1, 1)
    net.connect(md, 0, rec, 0, 8, n_tiles, T * n_tiles)
    net.connect(md, 1, cnt, 0, 4, 1, T + 1)
    net.finalize()
    return net, src, rec, cnt, n_tiles


def bench_motion(args, P, torch, pk, ws):
    from paper_1611_03226_b300 import _lib as L
    T = 300 if not args.quick else 60
    w = synth.motion(n_frames=T)
    H, W = w.height, w.width
    frames = np.stack(gen_parallel(w.frame, T))
    host = torch.from_numpy(frames).pin_memory()
    dev = host.to("cuda")
    net, src, rec, cnt, n_tiles = motion_net(P, torch, T, H, W)
    rec_dev = torch.empty(T * n_tiles * 8, dtype=torch.uint8, device="cuda")
    cnt_dev = torch.empty(T * 4, dtype=torch.uint8, device="cuda")
    l2 = torch.empty((2, 256 << 20), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def one_step(timed, evs):
        net.push(src, dev)
        flush_l2(l2)
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.run_async(1, L.DF_RUN_GRAPH)
            e1.record(stream)
            evs.append((e0, e1))
        else:
            net.run_async(1, L.DF_RUN_GRAPH)
        fired = net.sync()
        _, nrec = net.pop(rec, out=rec_dev)
        _, ncnt = net.pop(cnt, out=cnt_dev)
        return nrec, ncnt, fired

    for _ in range(args.warmup):
        one_step(False, None)
    evs = []
    barrier(ws)
    torch.cuda.synchronize()
    fired0 = net.sync()
    recs = 0
    for _ in range(args.steps):
        nrec, ncnt, _ = one_step(True, evs)
        assert ncnt == T
        recs += nrec
    torch.cuda.synchronize()
    fired = net.sync() - fired0
    assert fired == T * args.steps, fired
    # duration of the dominant kernel: the same steps launched eagerly with event timing
    net.profile(True)
    for _ in range(args.steps):
        net.push(src, dev)
        flush_l2(l2)
        net.run_async(1)
        net.sync()
        net.pop(rec, out=rec_dev)
        net.pop(cnt, out=cnt_dev)
    main_ms, main_n = net.profile_get(L.DF_PROF_MD_MAIN)
    step_ms, _ = net.profile_get(L.DF_PROF_STEP)
    net.profile(False)
    ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = max_over_ranks(statistics.mean(ms), ws)
    value = ws * T / (ms_step / 1e3)
    alg_bytes = T * W * H                        # each frame byte read once by the main kernel
    main_avg = main_ms / max(main_n, 1)
    achieved = alg_bytes / (main_avg / 1e3) / 1e9
    # end to end: push from pinned host memory, run, pop records + counts to host
    rec_h = np.empty(T * n_tiles * 8, np.uint8)
    cnt_h = np.empty(T * 4, np.uint8)
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.push(src, host)
        net.run(1)
        r = net.pop(rec, out=rec_h, dtype=np.uint64)
        c = net.pop(cnt, out=cnt_h, dtype=np.uint32)
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e.append((t1 - t0, len(r), len(c)))
    e2e_s = max_over_ranks(statistics.mean(x[0] for x in e2e), ws)
    net.close()
    return {
        "workload": f"motion_{T}x{W}x{H}", "value": value, "unit": "frames/s", "ms_per_step": ms_step,
        "dtype": "u8", "frames": T,
        "records_per_step": recs / args.steps,
        "kernel_ms": {"md_main_avg": main_avg, "eager_step_avg": step_ms / max(args.steps, 1)},
        "gpu_launches_per_step": 3,
        "launch_mode": "CUDA graph replay of one engine step (plan, main and emit kernels)",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"],
                     "traffic": profiled_traffic("k_md_main_tma__motion_300x1920x1080.md") if T == 300 else None,
                     "kernel": "k_md_main_tma", "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_source": pk["source"]},
        "e2e": {"value": ws * T / e2e_s, "unit": "frames/s",
                "h2d_bytes_per_step": T * W * H,
                "d2h_bytes_per_step": int(statistics.mean(x[1] for x in e2e)) * 8 + T * 4},
        "_oracle": (w, frames),
    }


def motion_cpu_baseline(w, frames, n=None):
    from oracle import motion as MD
    n = len(frames) if n is None else n
    T, H, W = frames.shape
    t0 = time.perf_counter()
    prev = np.zeros_like(frames[0])
    for t in range(n):
        MD.detect(frames[t], prev)
        prev = frames[t]
    dt = time.perf_counter() - t0
    host = host_info()
    run_s, done, procs = parallel_oracle(_motion_range, [(a, b, T, H, W) for a, b in split(T, host["nproc"])])
    return {"value": n / dt, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {len(frames)} frames, numpy single thread",
            "host": host,
            "threaded": threaded_motion(frames, H, W, min(n, 30)),
            "processes": {"value": done / run_s, "unit": "frames/s", "cores": procs,
                          "sample": f"all {T} frames in {procs} contiguous ranges, one oracle network per "
                                    "process (the frame before a range is its previous-frame initial token); "
                                    "time of the slowest process"}}


def dpd_flops(masks, M, L):
    pops = np.array([bin(int(m)).count("1") for m in masks])
    return float(8 * M * L * pops.sum())


def bench_dpd_large(args, P, torch, pk, ws):
    from paper_1611_03226_b300 import _lib as L
    nb = 512 if not args.quick else 64
    w = synth.dpd_large(n_blocks=nb)
    Lb = w.block_len
    blocks = gen_parallel(w.block, nb)
    host = torch.from_numpy(np.stack(blocks)).pin_memory()
    del blocks
    dev = host.to("cuda")
    masks_h = torch.from_numpy(w.masks.copy()).pin_memory()
    masks_d = masks_h.to("cuda")
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    c, d = net.add_source(), net.add_source()
    a = net.add_dpd(w.h, w.orders, Lb)
    s = net.add_sink()
    cap = nb + w.delay
    net.connect(c, 0, a, 0, 4, 1, cap)
    net.connect(d, 0, a, 1, Lb * 8, 1, cap, w.delay)
    net.connect(a, 0, s, 0, Lb * 8, 1, cap)
    net.finalize()
    out = torch.empty((nb + w.delay, Lb), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    # The d initial blocks stay in the data channel: each step fires exactly nb firings
    # (ctrl tokens limit), consuming the d zeros first, so the steady state carries the
    # last d blocks of one step into the next (a continuing stream).

    def step(timed, evs):
        net.push(c, masks_d)
        net.push(d, dev)
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.run_async(1)
            e1.record(stream)
            evs.append((e0, e1))
        else:
            net.run_async(1)
        net.sync()
        net.pop(s, out=out)

    for _ in range(args.warmup):
        step(False, None)
    evs = []
    barrier(ws)
    torch.cuda.synchronize()
    net.profile(True)
    f0 = net.sync()
    steps = max(3, args.steps // 4)
    for _ in range(steps):
        step(True, evs)
    torch.cuda.synchronize()
    assert net.sync() - f0 == nb * steps
    body_ms, body_n = net.profile_get(L.DF_PROF_DPD_BODY)
    net.profile(False)
    ms_step = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in evs), ws)
    samples = nb * Lb
    body_avg = body_ms / max(body_n, 1)
    flops = dpd_flops(w.masks, w.n_taps, Lb)
    peak_tf, n_sm = fp32_peak(pk, torch)
    achieved_tf = flops / (body_avg / 1e3) / 1e12
    hbm_gbs = 16.0 * samples / (body_avg / 1e3) / 1e9
    # e2e through the C ABI from pinned host memory (blocks in, blocks out)
    out_h = torch.empty((nb + w.delay, Lb), dtype=torch.complex64).pin_memory()
    e2e = []
    for i in range(1 + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.push(c, masks_h)
        net.push(d, host)
        net.run(1)
        net.pop(s, out=out_h)
        if i >= 1:
            e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e), ws)
    net.close()
    return {
        "workload": f"dpd_large_{nb}x{Lb}", "value": ws * samples / (ms_step / 1e3) / 1e6,
        "unit": "Msamples/s", "ms_per_step": ms_step, "dtype": "f32",
        "kernel_ms": {"dpd_body_avg": body_avg},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": achieved_tf / peak_tf,
                     "traffic": profiled_traffic("k_dpd_body__dpd_large_512x1048576.md") if nb == 512 else None,
                     "kernel": "k_dpd_body",
                     "algorithmic_flops_per_launch": flops,
                     "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x sm_max_mhz",
                     "hbm": {"achieved": hbm_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                             "frac": hbm_gbs / pk["hbm_gbs"], "bytes_per_sample": 16}},
        "e2e": {"value": ws * samples / e2e_s / 1e6, "unit": "Msamples/s",
                "h2d_bytes_per_step": samples * 8 + nb * 4, "d2h_bytes_per_step": samples * 8},
        "gpu_launches_per_step": 2,
        "_oracle": w,
    }


def dpd_cpu_baseline(w, n_blocks):
    from oracle import nets as ON
    net, ids = ON.dpd_fused(w.h, w.orders, w.block_len, w.delay, n_blocks + w.delay)
    net.push(ids["ctrl"], ON.as_tokens_ctrl(w.masks[:n_blocks]))
    net.push(ids["data"], ON.as_tokens_blocks(w.blocks(0, n_blocks)))
    t0 = time.perf_counter()
    net.run(-1)
    dt = time.perf_counter() - t0
    host = host_info()
    run_s, done, procs = parallel_oracle(_dpd_large_range, split(3 * host["nproc"], host["nproc"]))
    # the paper's Poly -> FIR_k -> Adder network with one thread per actor (Sec. 3.3)
    nt = 4
    tnet, tids = ON.dpd_expanded(w.h, w.orders, w.block_len, w.delay, nt + w.delay)
    tnet.push(tids["ctrl"], ON.as_tokens_ctrl(w.masks[:nt]))
    tnet.push(tids["data"], ON.as_tokens_blocks(w.blocks(0, nt)))
    t0 = time.perf_counter()
    tnet.run_threaded()
    tdt = time.perf_counter() - t0
    return {"value": n_blocks * w.block_len / dt / 1e6, "unit": "Msamples/s", "cores": 1,
            "kind": "oracle",
            "sample": f"first {n_blocks} of {w.n_blocks} blocks, float64 numpy single thread",
            "host": host,
            "threaded": {"value": nt * w.block_len / tdt / 1e6, "unit": "Msamples/s",
                         "threads": w.n_branches + 2,
                         "sample": f"first {nt} blocks through Poly, {w.n_branches} FIRs and Adder, one "
                                   "thread per actor"},
            "processes": {"value": done / run_s / 1e6, "unit": "Msamples/s", "cores": procs,
                          "sample": f"{3 * procs} blocks as {procs} independent 3-block streams, one per process; "
                                    "time of the slowest process"}}


def bench_dpd_tiny(args, P, torch, pk):
    from paper_1611_03226_b300 import _lib as L
    w = synth.dpd_tiny()
    Lb, nb = w.block_len, w.n_blocks
    dev = torch.from_numpy(w.blocks()).to("cuda")
    masks = torch.from_numpy(w.masks.copy()).to("cuda")
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    c, d = net.add_source(), net.add_source()
    a = net.add_dpd(w.h, w.orders, Lb)
    s = net.add_sink()
    net.connect(c, 0, a, 0, 4, 1, w.capacity)
    net.connect(d, 0, a, 1, Lb * 8, 1, w.capacity, w.delay)
    net.connect(a, 0, s, 0, Lb * 8, 1, w.capacity)
    net.finalize()
    out = torch.empty((w.capacity, Lb), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    chunk = w.capacity - w.delay
    # tile configuration from the autotuner on one step's worth of blocks (then drained)
    net.push(c, masks[:chunk])
    net.push(d, dev[:chunk])
    net.autotune()
    net.pop(s, out=out)
    tile = net.get_tile(a)

    def whole(flags):
        evs = []
        for i in range(0, nb, chunk):
            k = min(chunk, nb - i)
            net.push(c, masks[i:i + k])
            net.push(d, dev[i:i + k])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.run_async(1, flags)
            e1.record(stream)
            evs.append((e0, e1))
            net.sync()
            net.pop(s, out=out)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    modes = {"per_phase_kernels": 0, "graph_replay": L.DF_RUN_GRAPH, "persistent_kernel": L.DF_RUN_PERSISTENT,
             "persistent_kernel_graph": L.DF_RUN_PERSISTENT | L.DF_RUN_GRAPH}
    ms_mode = {}
    for name, flags in modes.items():
        for _ in range(args.warmup):
            whole(flags)
        ms_mode[name] = statistics.mean(whole(flags) for _ in range(args.steps))
    net.close()
    ms = min(ms_mode.values())
    return {"workload": f"dpd_tiny_{nb}x{Lb}_cap{w.capacity}", "value": nb * Lb / (ms / 1e3) / 1e6,
            "unit": "Msamples/s", "ms_per_step": ms, "dtype": "f32", "launch_modes_ms": ms_mode,
            "tile": {"samples": tile[0], "threads": tile[1], "source": "df_autotune"},
            "note": "device time of the 10 engine steps that stream 64 blocks through capacity-8 FIFOs"}


def bench_md_paper(args, P, torch, pk):
    """The paper's own motion pipeline (Sec. 4.1: Gauss -> Thres -> Med) on 320x240 frames at
    rate 4, all frames pushed before the step; one step fires every actor over all of them."""
    from paper_1611_03226_b300 import _lib as L
    T = 4096 if not args.quick else 512
    H, W, rate, thr = 240, 320, 4, 20
    w = synth.motion(n_frames=T, height=H, width=W)
    frames = np.stack(gen_parallel(w.frame, T))
    host = torch.from_numpy(frames).pin_memory()
    dev = host.to("cuda")
    out_dev = torch.empty_like(dev)
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    fb = H * W
    src, g, t, m, snk = (net.add_source(), net.add_gauss5(W, H), net.add_thres(W, H, thr),
                         net.add_med5(W, H), net.add_sink())
    cap = T + 1
    net.connect(src, 0, g, 0, fb, rate, cap)
    net.connect(g, 0, t, 0, fb, rate, cap)
    net.connect(g, 1, t, 1, fb, rate, cap, 1)
    net.connect(t, 0, m, 0, fb, rate, cap)
    net.connect(m, 0, snk, 0, fb, rate, cap)
    net.finalize()
    l2 = torch.empty((2, 256 << 20), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(timed, evs, flags):
        net.push(src, dev)
        flush_l2(l2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.run_async(1, flags)
        e1.record(stream)
        fired = net.sync()
        _, n = net.pop(snk, out=out_dev)
        if timed:
            evs.append((e0, e1))
        return n

    modes = {"graph": L.DF_RUN_GRAPH, "eager": 0}
    ms_mode = {}
    for name, flags in modes.items():
        for _ in range(args.warmup):
            step(False, None, flags)
        evs = []
        for _ in range(args.steps):
            assert step(True, evs, flags) == (T // rate) * rate
        torch.cuda.synchronize()
        ms_mode[name] = statistics.mean(a.elapsed_time(b) for a, b in evs)
    ms = min(ms_mode.values())
    frames_done = (T // rate) * rate
    # Gauss r + 2w, Thres r + w (its previous frames are its current frames one
    # token earlier, each read once), Med r + w
    bytes_per_frame = 7 * fb
    achieved = bytes_per_frame * frames_done / (ms / 1e3) / 1e9
    # end to end: pinned host frames in, motion maps out to pinned host memory
    out_h = torch.empty_like(host).pin_memory()
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.push(src, host)
        net.run(1)
        net.pop(snk, out=out_h.numpy())
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    net.close()
    # the paper's concurrent host actors: a producer thread pushes 256-frame
    # chunks from pinned memory and a consumer thread pops motion maps into
    # pinned memory, through channels of 1024 frames, while steps run
    from paper_1611_03226_b300.stream import stream
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    src, g, t, m, snk = (net.add_source(), net.add_gauss5(W, H), net.add_thres(W, H, thr),
                         net.add_med5(W, H), net.add_sink())
    cap_s, chunk = 1024, 256
    net.connect(src, 0, g, 0, fb, rate, cap_s)
    net.connect(g, 0, t, 0, fb, rate, cap_s)
    net.connect(g, 1, t, 1, fb, rate, cap_s, 1)
    net.connect(t, 0, m, 0, fb, rate, cap_s)
    net.connect(m, 0, snk, 0, fb, rate, cap_s)
    net.finalize()
    pop_buf = torch.empty((chunk, H, W), dtype=torch.uint8).pin_memory()
    st_py, st_s = [], []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got, _ = stream(net, {src: [host[j:j + chunk] for j in range(0, T, chunk)]},
                        {snk: (chunk, pop_buf)}, flags=L.DF_RUN_GRAPH)
        dt = time.perf_counter() - t0
        assert got[snk] == frames_done
        if i >= args.warmup:
            st_py.append(dt)
    # the same with the native runner (C++ threads, df_stream)
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got, _ = net.stream({src: (host, chunk)}, {snk: (out_h, chunk)}, L.DF_RUN_GRAPH)
        dt = time.perf_counter() - t0
        assert got[snk] == frames_done
        if i >= args.warmup:
            st_s.append(dt)
    net.close()
    # the paper's own buffers (Sec. 3.2): Eq. 1 sizes every channel (8-frame
    # double buffers, a 13-slot delay buffer with the Fig. 2 access pattern),
    # so the host threads push one window of 4 frames at a time
    T1 = min(T, 1024)
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    src, g, t, m, snk = (net.add_source(), net.add_gauss5(W, H), net.add_thres(W, H, thr),
                         net.add_med5(W, H), net.add_sink())
    chans = [net.connect(src, 0, g, 0, fb, rate, "eq1"), net.connect(g, 0, t, 0, fb, rate, "eq1"),
             net.connect(g, 1, t, 1, fb, rate, "eq1", 1), net.connect(t, 0, m, 0, fb, rate, "eq1"),
             net.connect(m, 0, snk, 0, fb, rate, "eq1")]
    net.finalize()
    eq1_bytes = sum(net.channel_info(c)["buffer_bytes"] for c in chans)
    st_q = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got, n_steps_eq1 = net.stream({src: (host[:T1], rate)}, {snk: (out_h[:T1], 2 * rate)}, L.DF_RUN_GRAPH)
        dt = time.perf_counter() - t0
        assert got[snk] == T1
        if i >= args.warmup:
            st_q.append(dt)
    net.close()
    # oracle on a bounded sample (64 frames)
    from oracle import motion_paper as MP
    from oracle import nets as ON
    ns = 64 if not args.quick else 16
    t0 = time.perf_counter()
    MP.pipeline(frames[:ns], thr)
    cpu_s = time.perf_counter() - t0
    host = host_info()
    nf = 64 * host["nproc"] if not args.quick else 16 * host["nproc"]
    run_s, done, procs = parallel_oracle(
        _md_paper_range, [(4 * a, 4 * b, T, H, W, thr) for a, b in split(nf // 4, host["nproc"])])
    tnet, tids = ON.motion_paper(H, W, ns + rate, rate, thr)
    tnet.push(tids["src"], list(frames[:ns]))
    t0 = time.perf_counter()
    tnet.run_threaded()
    thr_s = time.perf_counter() - t0
    return {"workload": f"md_paper_{T}x{W}x{H}_rate{rate}", "value": frames_done / (ms / 1e3),
            "unit": "frames/s", "ms_per_step": ms, "dtype": "u8", "launch_modes_ms": ms_mode,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": None,
                         "algorithmic_bytes_per_frame": bytes_per_frame,
                         "note": "whole step (3 plan and 3 body kernels) against its channel traffic"},
            "e2e": {"value": frames_done / statistics.mean(e2e), "unit": "frames/s",
                    "h2d_bytes_per_step": T * fb, "d2h_bytes_per_step": frames_done * fb},
            "e2e_streamed": {"value": frames_done / statistics.mean(st_s), "unit": "frames/s",
                             "python_threads_value": frames_done / statistics.mean(st_py),
                             "note": "native producer and consumer threads (df_stream) beside the running "
                                     "steps (DF_IO_CONCURRENT), 1024-frame channels, 256-frame chunks; "
                                     "python_threads_value: the same with Python threads"},
            "e2e_streamed_eq1": {"value": T1 / statistics.mean(st_q), "unit": "frames/s", "frames": T1,
                                 "steps": n_steps_eq1, "buffer_bytes": eq1_bytes,
                                 "paper_table1_MB": 3.46,
                                 "note": "native runner as e2e_streamed, but every channel sized by Eq. 1 "
                                         "(the paper's layout, Fig. 2 delay buffer): 4-frame pushes, "
                                         "8-frame pops"},
            "cpu_baseline": {"value": ns / cpu_s, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {ns} frames, numpy single thread", "host": host,
                             "threaded": {"value": ns / thr_s, "unit": "frames/s", "threads": 3,
                                          "sample": f"first {ns} frames; Gauss, Thres and Med one thread each "
                                                    "(Sec. 3.3)"},
                             "processes": {"value": done / run_s, "unit": "frames/s", "cores": procs,
                                           "sample": f"{done} frames in {procs} contiguous ranges, one oracle "
                                                     "network per process; time of the slowest process"}},
            "paper_table3_context": {"i7_gpu_fps": 6063, "carrizo_gpu_fps": 4614,
                                     "note": "Sec. 4.1, Table 3, other hardware (context only)"}}


def bench_dpd_batch(args, P, torch, pk):
    """256 independent channels (uneven lengths, taps and branch sets) with 16
    resident blocks each; one engine step fires all of them."""
    from paper_1611_03226_b300 import _lib as L
    w = synth.dpd_batch()
    C, nb = w.n_channels, w.blocks_per_channel
    pairs = [(c, b) for c in range(C) for b in range(nb)]
    blocks = gen_parallel(lambda i: w.block(*pairs[i]), len(pairs))
    dev = [torch.from_numpy(np.stack(blocks[c * nb:(c + 1) * nb])).to("cuda") for c in range(C)]
    del blocks
    masks = [torch.full((nb,), int(w.masks[c]), dtype=torch.int32, device="cuda") for c in range(C)]
    outs = [torch.empty_like(d) for d in dev]
    net = P.Net(stream=torch.cuda.current_stream().cuda_stream)
    ids = []
    for c in range(C):
        Lc = int(w.lengths[c])
        d = {"ctrl": net.add_source(), "data": net.add_source(),
             "dpd": net.add_dpd(w.h[c], w.orders, Lc), "sink": net.add_sink()}
        net.connect(d["ctrl"], 0, d["dpd"], 0, 4, 1, nb)
        net.connect(d["data"], 0, d["dpd"], 1, Lc * 8, 1, nb)
        net.connect(d["dpd"], 0, d["sink"], 0, Lc * 8, 1, nb)
        ids.append(d)
    net.finalize()
    stream = torch.cuda.current_stream()

    def push_all():
        for c in range(C):
            net.push(ids[c]["ctrl"], masks[c])
            net.push(ids[c]["data"], dev[c])

    def pop_all():
        for c in range(C):
            net.pop(ids[c]["sink"], out=outs[c])

    push_all()
    assert net.autotune() == C * nb
    pop_all()
    tuned = net.get_tile(ids[0]["dpd"])

    def timed(flags, steps):
        ms = []
        for i in range(args.warmup + steps):
            push_all()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.run_async(1, flags)
            e1.record(stream)
            assert net.sync() >= 0
            pop_all()
            if i >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms)

    steps = max(3, args.steps // 4)
    t_graph = timed(L.DF_RUN_GRAPH, steps)
    t_eager = timed(0, steps)
    t_per = timed(L.DF_RUN_NO_BATCH, steps)
    t_per_graph = timed(L.DF_RUN_NO_BATCH | L.DF_RUN_GRAPH, steps)
    t_pers = timed(L.DF_RUN_PERSISTENT, steps)
    t_pers_graph = timed(L.DF_RUN_PERSISTENT | L.DF_RUN_GRAPH, steps)
    # kernel time of the batched body
    push_all()
    net.profile(True)
    net.run(1)
    body_ms, _ = net.profile_get(L.DF_PROF_DPD_BODY)
    net.profile(False)
    pop_all()
    net.close()
    samples = int(w.lengths.sum()) * nb
    flops = float(sum(8 * int(w.taps[c]) * int(w.lengths[c]) * nb * bin(int(w.masks[c])).count("1")
                      for c in range(C)))
    peak_tf, _ = fp32_peak(pk, torch)
    ach = flops / (body_ms / 1e3) / 1e12
    # oracle on the first four channels
    from oracle import nets as ON
    t0 = time.perf_counter()
    n_cpu = 0
    for c in range(4):
        onet, oi = ON.dpd_fused(w.h[c], w.orders, int(w.lengths[c]), 0, nb)
        onet.push(oi["ctrl"], ON.as_tokens_ctrl([int(w.masks[c])] * nb))
        onet.push(oi["data"], ON.as_tokens_blocks([w.block(c, b) for b in range(nb)]))
        onet.run(-1)
        n_cpu += int(w.lengths[c]) * nb
    cpu_s = time.perf_counter() - t0
    host = host_info()
    run_s, done, procs = parallel_oracle(_dpd_batch_channel, list(range(min(C, host["nproc"]))))
    return {
        "workload": f"dpd_batch_{C}ch_x{nb}blocks", "value": samples / (t_graph / 1e3) / 1e6,
        "unit": "Msamples/s", "ms_per_step": t_graph, "dtype": "f32", "samples_per_step": samples,
        "launch_modes_ms": {"batched_graph": t_graph, "batched_eager": t_eager,
                            "per_channel_eager": t_per, "per_channel_graph": t_per_graph,
                            "persistent": t_pers, "persistent_graph": t_pers_graph},
        "persistent_note": "one cooperative launch runs the step (plans, grid barrier, bodies); "
                           "persistent_graph replays that launch from a CUDA graph",
        "batched_vs_per_channel": t_per / t_graph,
        "autotuned_tile": {"samples": tuned[0], "threads": tuned[1]},
        "gpu_launches_per_step": {"batched": 2, "per_channel": 2 * C},
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": ach / peak_tf,
                     "traffic": profiled_traffic("k_dpd_body__dpd_batch_256ch_x16blocks.md"),
                     "kernel": "k_dpd_body", "algorithmic_flops_per_launch": flops,
                     "algorithmic_bytes_per_launch": 16 * samples},
        "cpu_baseline": {"value": n_cpu / cpu_s / 1e6, "unit": "Msamples/s", "cores": 1,
                         "kind": "oracle", "sample": "channels 0-3, 16 blocks each", "host": host,
                         "processes": {"value": done / run_s / 1e6, "unit": "Msamples/s", "cores": procs,
                                       "sample": f"channels 0-{procs - 1}, one per process; time of the "
                                                 "slowest process"}},
    }


def bench_dpd_fit(args, P, torch, pk):
    """Indirect-learning fit: 2^18 samples, 4 branches x 10 taps, 200 Adam steps."""
    from paper_1611_03226_b300 import dpd as G
    from paper_1611_03226_b300 import fit as F
    w = synth.dpd_fit()
    x = torch.from_numpy(w.x).to("cuda")
    n = x.numel()
    stream = torch.cuda.current_stream()
    F.ila_fit(x, steps=3)                                   # warm-up
    F.ila_fit(x, steps=3, graph=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h, losses = F.ila_fit(x, steps=w.steps, lr=w.lr)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fit = e0.elapsed_time(e1)
    # the same fit with the training step issued eagerly (no graph)
    e0.record(stream)
    F.ila_fit(x, steps=w.steps, lr=w.lr, graph=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fit_eager = e0.elapsed_time(e1)
    gain = F.small_signal_gain()
    nmse_off = F.nmse_db(F.saleh_pa(x) / gain, x)
    nmse_on = F.nmse_db(F.saleh_pa(G.dpd_forward(x, h, w.orders)) / gain, x)
    # forward and adjoint kernels alone
    u = (F.saleh_pa(x) / gain).to(torch.complex64).contiguous()
    gy = torch.randn_like(u)

    def avg(fn, reps=20):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    fwd_ms = avg(lambda: G.dpd_forward(u, h, w.orders))
    bwd_ms = avg(lambda: G.dpd_backward(u, h, w.orders, gy))
    # iterative indirect learning (predistorter in the loop), 3 iterations of the same fit
    t0 = time.perf_counter()
    _, _, nmse_iter = F.ila_fit_iterative(x, iterations=3, steps=w.steps, lr=w.lr)
    torch.cuda.synchronize()
    iter_s = time.perf_counter() - t0
    # the same forward through a one-block engine network (all branches active)
    net = P.Net(stream=stream.cuda_stream)
    c, d = net.add_source(), net.add_source()
    a = net.add_dpd(h.cpu().numpy(), w.orders, n)
    s = net.add_sink()
    net.connect(c, 0, a, 0, 4, 1, 1)
    net.connect(d, 0, a, 1, n * 8, 1, 1)
    net.connect(a, 0, s, 0, n * 8, 1, 1)
    net.finalize()
    mask = torch.full((1,), 15, dtype=torch.int32, device="cuda")
    out = torch.empty_like(u)

    def engine_fwd():
        net.push(c, mask)
        net.push(d, u)
        net.run_async(1)
        net.sync()
        net.pop(s, out=out)

    eng_ms = []
    for i in range(6):
        net.push(c, mask)
        net.push(d, u)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        net.run_async(1)
        a1.record(stream)
        net.sync()
        net.pop(s, out=out)
        if i >= 2:
            eng_ms.append(a0.elapsed_time(a1))
    engine_ms = statistics.mean(eng_ms)
    # the network continues each branch's FIR history across blocks; the
    # stateless operator starts from zeros, so compare past the first M-1 samples
    ref = G.dpd_forward(u, h, w.orders)
    m0 = w.n_taps - 1
    err = float((out[m0:] - ref[m0:]).abs().norm() / ref[m0:].abs().norm())
    net.close()
    # oracle: 10 float64 steps on the same signal
    from oracle import fit as OF
    t0 = time.perf_counter()
    OF.ila_fit(w.x, steps=10, lr=w.lr)
    cpu_ms = (time.perf_counter() - t0) / 10 * 1e3
    return {
        "workload": f"dpd_fit_{n}_K4_M10_{w.steps}steps", "value": ms_fit / w.steps,
        "unit": "ms/Adam step", "higher_is_better": False, "dtype": "f32",
        "launch_mode": "one CUDA graph per training step (forward, loss, adjoint, Adam update)",
        "eager_ms_per_step": ms_fit_eager / w.steps,
        "fwd_bwd_msamples_s": n / ((fwd_ms + bwd_ms) / 1e3) / 1e6,
        "kernel_ms": {"forward": fwd_ms, "backward": bwd_ms},
        "loss_first_last": [float(losses[0]), float(losses[-1])],
        "nmse_db": {"without_dpd": nmse_off, "with_dpd": nmse_on},
        "iterative_ila": {"iterations": 3, "nmse_db_after_each": [float(v) for v in nmse_iter],
                          "seconds": iter_s,
                          "note": "predistorter in the loop; at this drive level the peaks reach "
                                  "saturation and further iterations lose linearity"},
        "engine_network_forward_ms": engine_ms, "engine_vs_stateless_rel_l2": err,
        "cpu_baseline": {"value": cpu_ms, "unit": "ms/Adam step", "cores": 1, "kind": "oracle",
                         "sample": "10 float64 steps of the 2^18-sample fit"},
    }


# --------------------------------------------------------------- arms ----
def gpu_arm(args):
    ws, rank, local = dist_setup(args)
    if rank == 0:
        oracle_pool()            # spawned before this process touches the GPU
    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    import paper_1611_03226_b300 as P
    pk = peaks()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    # The engine runs on this (non-default) stream; torch's timing events are
    # recorded on the same stream.
    work = torch.cuda.Stream()
    extra = {}
    want = set(args.only.split(",")) if args.only else set(SECONDARY)
    with torch.cuda.stream(work):
        md = bench_motion(args, P, torch, pk, ws)
        if "dpd_large" in want:
            extra["dpd_large"] = bench_dpd_large(args, P, torch, pk, ws)
        if ws == 1:
            if "dpd_tiny" in want:
                extra["dpd_tiny"] = bench_dpd_tiny(args, P, torch, pk)
            if "dpd_batch" in want and not args.quick:
                extra["dpd_batch"] = bench_dpd_batch(args, P, torch, pk)
            if "dpd_fit" in want:
                extra["dpd_fit"] = bench_dpd_fit(args, P, torch, pk)
            if "md_paper" in want:
                extra["md_paper"] = bench_md_paper(args, P, torch, pk)
    clocks = sampler.stop() if rank == 0 else None
    if rank != 0:
        return
    w, frames = md.pop("_oracle")
    cpu = motion_cpu_baseline(w, frames)
    if "dpd_large" in extra:
        wl = extra["dpd_large"].pop("_oracle")
        extra["dpd_large"]["cpu_baseline"] = dpd_cpu_baseline(wl, 8 if args.quick else 24)
    line = {
        "metric": METRIC, "value": md["value"], "unit": md["unit"], "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": md["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; textured background, moving rectangles, clipped noise)",
        "config": {"workload": md["workload"], "frames": md["frames"], "width": 1920, "height": 1080,
                   "threshold": 25, "tile": 16, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "inputs": "resident in HBM; re-pushed device-to-device before each step (untimed)",
                   "l2": "before every timed step a 256 MB buffer is written and a second 256 MB buffer read (L2 holds no frame data and no dirty lines); frames (622 MB) exceed L2"},
        "roofline": md["roofline"], "cpu_baseline": cpu, "e2e": md["e2e"],
        "gpu_launches": md["gpu_launches_per_step"] * args.steps,
        "kernel_ms": md["kernel_ms"], "records_per_step": md["records_per_step"],
        "launch_mode": md["launch_mode"],
        "clocks": clocks, "workloads": extra,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def reference_arm(args):
    """The oracle on the host's cores over the whole headline workload: every
    step runs the 300 frames as contiguous ranges, one unmodified oracle
    network per spawned process (the frame before a range is its
    previous-frame initial token); a step's time is the slowest process's run."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    T = 300 if not args.quick else 60
    H, W = 1080, 1920
    host = host_info()
    parts = [(a, b, T, H, W) for a, b in split(T, host["nproc"])]
    times = []
    for i in range(args.warmup + args.steps):
        run_s, done, procs = parallel_oracle(_motion_range, parts)
        assert done == T
        if i >= args.warmup:
            times.append(run_s)
    ms = 1e3 * statistics.mean(times)
    value = T / (ms / 1e3)
    sample = (f"all {T} frames of the 1920x1080 workload per step, {procs} contiguous ranges, one oracle "
              f"network per process on {procs} host cores ({host['cpu_model']}); time of the slowest process")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": f"motion_{T}x{W}x{H}", "frames": T, "width": W,
                                            "height": H, "threshold": 25, "tile": 16, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": procs, "kind": "oracle",
                             "sample": sample, "host": host},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(args):
    """--case NAME: that workload's engine network alone, args.warmup + args.steps
    eager steps of push, run(1), pop (no headline, no CPU baselines, no JSON line).
    The ncu summaries under profiles/ are taken on this command, the kernel
    filtered by name and the warm-up launches skipped (-s)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1611_03226_b300 as P
    work = torch.cuda.Stream()
    with torch.cuda.stream(work):
        net = P.Net(stream=work.cuda_stream)
        if args.case == "dpd_large":
            nb = args.case_blocks
            w = synth.dpd_large(n_blocks=nb)
            Lb = w.block_len
            dev = torch.from_numpy(np.stack(gen_parallel(w.block, nb))).to("cuda")
            masks = torch.from_numpy(w.masks.copy()).to("cuda")
            c, d, a, s = net.add_source(), net.add_source(), net.add_dpd(w.h, w.orders, Lb), net.add_sink()
            net.connect(c, 0, a, 0, 4, 1, nb + w.delay)
            net.connect(d, 0, a, 1, Lb * 8, 1, nb + w.delay, w.delay)
            net.connect(a, 0, s, 0, Lb * 8, 1, nb + w.delay)
            net.finalize()
            net.set_tile(a, 4096, 256)
            out = torch.empty((nb + w.delay, Lb), dtype=torch.complex64, device="cuda")
            push = lambda: (net.push(c, masks), net.push(d, dev))
            pop = lambda: net.pop(s, out=out)
        elif args.case == "dpd_batch":
            w = synth.dpd_batch()
            C, nb = w.n_channels, w.blocks_per_channel
            pairs = [(ch, b) for ch in range(C) for b in range(nb)]
            blocks = gen_parallel(lambda i: w.block(*pairs[i]), len(pairs))
            dev = [torch.from_numpy(np.stack(blocks[ch * nb:(ch + 1) * nb])).to("cuda") for ch in range(C)]
            masks = [torch.full((nb,), int(w.masks[ch]), dtype=torch.int32, device="cuda") for ch in range(C)]
            outs = [torch.empty_like(x) for x in dev]
            ids = []
            for ch in range(C):
                Lc = int(w.lengths[ch])
                ids.append((net.add_source(), net.add_source(), net.add_dpd(w.h[ch], w.orders, Lc), net.add_sink()))
                cs, ds, a, sk = ids[-1]
                net.connect(cs, 0, a, 0, 4, 1, nb)
                net.connect(ds, 0, a, 1, Lc * 8, 1, nb)
                net.connect(a, 0, sk, 0, Lc * 8, 1, nb)
            net.finalize()
            for cs, ds, a, sk in ids:
                net.set_tile(a, 4096, 256)

            def push():
                for ch, (cs, ds, a, sk) in enumerate(ids):
                    net.push(cs, masks[ch])
                    net.push(ds, dev[ch])

            def pop():
                for ch, (cs, ds, a, sk) in enumerate(ids):
                    net.pop(sk, out=outs[ch])
        else:                                      # md_paper
            T, H, W, rate, thr = 4096, 240, 320, 4, 20
            wm = synth.motion(n_frames=T, height=H, width=W)
            dev = torch.from_numpy(np.stack(gen_parallel(wm.frame, T))).to("cuda")
            out = torch.empty_like(dev)
            src, g, t, m, snk = (net.add_source(), net.add_gauss5(W, H), net.add_thres(W, H, thr),
                                 net.add_med5(W, H), net.add_sink())
            fb = H * W
            net.connect(src, 0, g, 0, fb, rate, T + 1)
            net.connect(g, 0, t, 0, fb, rate, T + 1)
            net.connect(g, 1, t, 1, fb, rate, T + 1, 1)
            net.connect(t, 0, m, 0, fb, rate, T + 1)
            net.connect(m, 0, snk, 0, fb, rate, T + 1)
            net.finalize()
            push = lambda: net.push(src, dev)
            pop = lambda: net.pop(snk, out=out)
        ms = []
        for i in range(args.warmup + args.steps):
            push()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            net.run(1)
            ms.append(1e3 * (time.perf_counter() - t0))
            pop()
        net.close()
    print(f"{args.case}: {args.steps} steps after {args.warmup} warm-up, host-timed step "
          f"{statistics.mean(ms[args.warmup:]):.3f} ms")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--quick", action="store_true", help="smaller workloads (smoke runs)")
    ap.add_argument("--only", default=None,
                    help="comma-separated secondary workloads to run besides the motion headline "
                         "(dpd_large, dpd_tiny, dpd_batch, dpd_fit, md_paper; 'motion' = none)")
    ap.add_argument("--case", default=None, choices=["dpd_large", "dpd_batch", "md_paper"],
                    help="run one workload's network alone for a profiler capture (no JSON line)")
    ap.add_argument("--case-blocks", type=int, default=64, help="blocks of the dpd_large case")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.case:
        profile_case(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
