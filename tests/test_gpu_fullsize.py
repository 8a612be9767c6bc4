"""Parity at the benchmark sizes and launch configurations.

* Large predistorter: 512 blocks of 2^20 samples (K <= 8, M = 16, two delay
  blocks) pushed whole and run once, the bench's launch; every block in which
  some branch becomes active again after two or more blocks without it (its
  FIR history then comes from a block further back), the first and last
  blocks and 64 more chosen at random, each against the float64 oracle.
* Batched predistorter: the bench's 256-channel network (lengths 1-256 Ki,
  16 blocks per channel, autotuned tile, then a CUDA-graph replay of a second
  step), every block of every channel against the oracle.
* Adjoint at the fit size (2^18), one past it, and 3 * 2^20 + 17 samples (tile
  partial sums beyond 256 per tap, strided grid).
* The allocating adjoint from two threads on two streams with different sizes.
* Valid frame widths the kernels do not implement are refused with DF_ENOTSUP.

The oracle runs on the host's cores in threads (numpy releases the GIL in its
array loops)."""
import ctypes
import os
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import dpd as D

pytestmark = pytest.mark.gpu

TOL = 1e-5
WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def P():
    import paper_1611_03226_b300 as P
    return P


def gap_blocks(masks, K):
    """Blocks in which some active branch was last active three or more blocks
    earlier (or never)."""
    last = [-(1 << 30)] * K
    out = []
    for i, m in enumerate(masks):
        hit = False
        for k in range(K):
            if (int(m) >> k) & 1:
                hit = hit or i - last[k] >= 3
                last[k] = i
        if hit:
            out.append(i)
    return out


@pytest.mark.slow
def test_large_workload_gap_and_random_blocks(P):
    import torch
    w = synth.dpd_large()
    L, n, d, M, K = w.block_len, w.n_blocks, w.delay, w.n_taps, w.n_branches
    enet, ei = EN.dpd_fused(P.Net, w.h, w.orders, L, d, n + d)
    enet.push(ei["ctrl"], np.ascontiguousarray(w.masks))
    with ThreadPoolExecutor(WORKERS) as ex:
        for b in range(0, n, 32):
            blocks = list(ex.map(w.block, range(b, min(n, b + 32))))
            enet.push(ei["data"], np.ascontiguousarray(np.stack(blocks)))
    assert enet.run(-1) == n
    out = torch.empty((n, L), dtype=torch.complex64, device="cuda")
    _, got = enet.pop(ei["sink"], out=out)
    assert got == n
    for key in ("ch_ctrl", "ch_data", "ch_out"):
        p, c, o = enet.counters(ei[key])
        assert p + (d if key == "ch_data" else 0) == c + o
    enet.close()
    rng = np.random.default_rng(3)
    check = set(gap_blocks(w.masks, K)) | {0, 1, 2, 3, n - 2, n - 1}
    check |= set(int(i) for i in rng.choice(n, 64, replace=False))
    assert len(check) > 300
    # input block i of the stream is data block i - d (zeros before)
    with ThreadPoolExecutor(WORKERS) as ex:
        tails = dict(zip(range(n), ex.map(lambda b: w.block(b)[L - (M - 1):], range(n))))

    def oracle_block(i):
        xi = np.zeros(L, np.complex64) if i < d else w.block(i - d)
        y = np.zeros(L, np.complex128)
        for k in range(K):
            if not (int(w.masks[i]) >> k) & 1:
                continue
            prev = [j for j in range(i) if (int(w.masks[j]) >> k) & 1]
            tail = tails[prev[-1] - d] if prev and prev[-1] >= d else np.zeros(M - 1, np.complex64)
            yk, _ = D.fir(w.h[k], D.psi(tail, w.orders[k]), D.psi(xi, w.orders[k]))
            y += yk
        return i, y

    errs = {}
    with ThreadPoolExecutor(WORKERS) as ex:
        for i, ref in ex.map(oracle_block, sorted(check)):
            errs[i] = D.rel_l2(out[i].cpu().numpy(), ref)
    worst = max(errs, key=errs.get)
    assert errs[worst] <= TOL, (worst, errs[worst])


@pytest.mark.slow
def test_batched_256_channels_bench_configuration(P):
    """Bench launch configuration of the batched workload: the autotuner's step,
    then a second step replayed from a CUDA graph; each channel's FIR histories
    continue from the first step into the second."""
    import torch
    from paper_1611_03226_b300 import _lib as Lb
    w = synth.dpd_batch()
    C, nb = w.n_channels, w.blocks_per_channel
    chans = [(w.h[c], w.orders, int(w.lengths[c])) for c in range(C)]
    net, ids = EN.dpd_batch(P.Net, chans, nb)
    with ThreadPoolExecutor(WORKERS) as ex:
        xs = list(ex.map(lambda c: np.stack([w.block(c, b) for b in range(nb)]), range(C)))
    dev = [torch.from_numpy(x).cuda() for x in xs]
    masks = [torch.full((nb,), int(w.masks[c]), dtype=torch.int32, device="cuda") for c in range(C)]
    torch.cuda.synchronize()          # the network's own stream reads these

    def push_all():
        for c in range(C):
            net.push(ids[c]["ctrl"], masks[c])
            net.push(ids[c]["data"], dev[c])

    def pop_all():
        outs = []
        for c in range(C):
            o = torch.empty_like(dev[c])
            _, got = net.pop(ids[c]["sink"], out=o)
            assert got == nb
            outs.append(o)
        return outs

    push_all()
    assert net.autotune() == C * nb
    tile = net.get_tile(ids[0]["dpd"])
    assert tile[0] > 0
    out1 = pop_all()
    push_all()
    assert net.run(1, Lb.DF_RUN_GRAPH) == C * nb
    out2 = pop_all()
    net.close()

    def check(c):
        L, M = int(w.lengths[c]), int(w.taps[c])
        s = xs[c].reshape(-1)
        y1 = np.zeros(s.size, np.complex128)
        y2 = np.zeros(s.size, np.complex128)
        for k in range(len(w.orders)):
            if not (int(w.masks[c]) >> k) & 1:
                continue
            z = D.psi(s, w.orders[k])
            a, hist = D.fir(w.h[c][k], np.zeros(M - 1, np.complex128), z)
            b, _ = D.fir(w.h[c][k], hist, z)
            y1 += a
            y2 += b
        e1 = max(D.rel_l2(out1[c][b].cpu().numpy(), y1[b * L:(b + 1) * L]) for b in range(nb))
        e2 = max(D.rel_l2(out2[c][b].cpu().numpy(), y2[b * L:(b + 1) * L]) for b in range(nb))
        return c, max(e1, e2)

    with ThreadPoolExecutor(WORKERS) as ex:
        errs = dict(ex.map(check, range(C)))
    worst = max(errs, key=errs.get)
    assert errs[worst] <= TOL, (worst, errs[worst], tile)


@pytest.mark.parametrize("n", [1 << 18, (1 << 18) + 1, 3 * (1 << 20) + 17])
def test_adjoint_at_fit_size_and_beyond(P, n):
    import torch
    from paper_1611_03226_b300 import dpd as G
    from paper_1611_03226_b300 import _lib as Lb
    rng = np.random.default_rng(n)
    K, M, orders = 4, 10, (1, 3, 5, 7)
    x = (rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    h[0, 0] = 1
    g = (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)
    xt, ht, gt = (torch.from_numpy(a).cuda() for a in (x, h, g))
    y = G.dpd_forward(xt, ht, orders).cpu().numpy()
    assert D.rel_l2(y, D.dpd_stream(x, h, orders)) <= TOL
    gx, gh = G.dpd_backward(xt, ht, orders, gt)
    rx, rh = D.dpd_stream_backward(x, h, orders, g)
    assert D.rel_l2(gx.cpu().numpy(), rx) <= 1e-3
    assert D.rel_l2(gh.cpu().numpy(), rh) <= 1e-3
    # the library-scratch entry point gives the same bits as the caller-scratch one
    gx2, gh2 = torch.empty_like(xt), torch.empty_like(ht)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    o = (ctypes.c_int32 * K)(*orders)
    assert Lb.lib.df_dpd_backward(p(xt), n, p(ht), K, M, o, p(gt), p(gx2), p(gh2),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    assert torch.equal(gx, gx2) and torch.equal(gh, gh2)


def test_allocating_adjoint_two_threads_two_streams(P):
    """Two threads call df_dpd_backward on streams of their own with different
    sizes, three times each, at the same time; every call gives the gradients
    of a call made alone."""
    import torch
    from paper_1611_03226_b300 import _lib as Lb
    K, M, orders = 4, 10, (1, 3, 5, 7)
    o = (ctypes.c_int32 * K)(*orders)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    cases = []
    for n in (50_000, 700_000):
        rng = np.random.default_rng(n)
        x = torch.from_numpy((rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64)).cuda()
        h = torch.from_numpy((rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)).cuda()
        g = torch.from_numpy((rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)).cuda()
        s0 = torch.cuda.Stream()
        gx, gh = torch.empty_like(x), torch.empty_like(h)
        torch.cuda.synchronize()
        assert Lb.lib.df_dpd_backward(p(x), n, p(h), K, M, o, p(g), p(gx), p(gh), ctypes.c_void_p(s0.cuda_stream)) == 0
        s0.synchronize()
        # the threads use fresh streams: their first calls grow scratch at the same time
        cases.append((n, x, h, g, torch.cuda.Stream(), gx.clone(), gh.clone()))
    results = [[] for _ in cases]

    def worker(i):
        n, x, h, g, s, _, _ = cases[i]
        for _ in range(3):
            gx, gh = torch.empty_like(x), torch.empty_like(h)
            st = Lb.lib.df_dpd_backward(p(x), n, p(h), K, M, o, p(g), p(gx), p(gh), ctypes.c_void_p(s.cuda_stream))
            results[i].append((st, gx, gh))
        s.synchronize()

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i, (_, _, _, _, _, gx_ref, gh_ref) in enumerate(cases):
        assert len(results[i]) == 3
        for st, gx, gh in results[i]:
            assert st == 0
            assert torch.equal(gx, gx_ref) and torch.equal(gh, gh_ref)


def test_adjoint_scratch_growth_refused_during_capture(P):
    """A call that would have to grow the library's scratch while its stream is
    being captured returns DF_ESTATE and enqueues nothing."""
    import torch
    from paper_1611_03226_b300 import _lib as Lb
    K, M, orders = 2, 5, (1, 3)
    o = (ctypes.c_int32 * K)(*orders)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    n = 1 << 21
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    h = torch.zeros((K, M), dtype=torch.complex64, device="cuda")
    gx, gh = torch.empty_like(x), torch.empty_like(h)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        st = Lb.lib.df_dpd_backward(p(x), n, p(h), K, M, o, p(x), p(gx), p(gh), ctypes.c_void_p(s.cuda_stream))
    assert st == Lb.DF_ESTATE


def test_unsupported_frame_widths_are_refused(P):
    from paper_1611_03226_b300 import _lib as Lb
    net = P.Net()
    for add, args in ((net.add_md, (1000, 64, 25)), (net.add_md, (48, 64, 25)),
                      (net.add_gauss5, (2064, 16)), (net.add_thres, (1000, 16, 20)), (net.add_med5, (24, 8))):
        with pytest.raises(Lb.DfError) as e:
            add(*args)
        assert e.value.status == Lb.DF_ENOTSUP, (add.__name__, args)
    for add, args in ((net.add_md, (0, 64, 25)), (net.add_gauss5, (-16, 8))):
        with pytest.raises(Lb.DfError) as e:
            add(*args)
        assert e.value.status == Lb.DF_EINVAL
    net.close()
