"""Host actors in threads of their own (the paper's concurrent host / GPU
execution): producer threads push, consumer threads pop and the test thread
runs steps, all at once; the output streams equal the oracle's."""
import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import motion as MD
from oracle import motion_paper as MP
from oracle import nets as ON

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1611_03226_b300 as P
    return P


def batches(arr, sizes_seed, lo=1, hi=3):
    rng = np.random.default_rng(sizes_seed)
    i = 0
    while i < len(arr):
        k = int(rng.integers(lo, hi + 1))
        yield np.ascontiguousarray(arr[i:i + k])
        i += k


@pytest.mark.parametrize("flags", ["per_phase", "graph", "persistent"])
def test_streamed_predistorter(P, flags):
    from paper_1611_03226_b300 import _lib as L
    from paper_1611_03226_b300.stream import stream
    fl = {"per_phase": 0, "graph": L.DF_RUN_GRAPH, "persistent": L.DF_RUN_PERSISTENT}[flags]
    w = synth.dpd_tiny()
    n, Lb = 40, w.block_len
    x, masks = w.blocks(0, n), np.ascontiguousarray(w.masks[:n])
    net, ids = EN.dpd_fused(P.Net, w.h, w.orders, Lb, w.delay, w.capacity)
    out, steps = stream(net, {ids["ctrl"]: batches(masks, 1), ids["data"]: batches(x, 2)},
                        {ids["sink"]: 3}, flags=fl)
    got = np.concatenate(out[ids["sink"]]).view(np.complex64).reshape(-1, Lb)
    net.close()
    onet, oi = ON.dpd_fused(w.h, w.orders, Lb, w.delay, n + w.delay)
    onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks))
    onet.push(oi["data"], ON.as_tokens_blocks(x))
    onet.run(-1)
    want = np.array(onet.pop(oi["sink"]))
    assert got.shape == want.shape == (n, Lb)
    for i in range(n):
        assert np.linalg.norm(got[i] - want[i]) <= 1e-5 * max(np.linalg.norm(want[i]), 1e-30)


def test_streamed_paper_pipeline(P):
    from paper_1611_03226_b300.stream import stream
    T, H, W, rate = 48, 240, 320, 4
    f = synth.motion(n_frames=T, height=H, width=W).frames()
    net, ids = EN.motion_paper(P.Net, H, W, 9, rate)
    out, _ = stream(net, {ids["src"]: batches(f, 3, 4, 4)}, {ids["sink"]: 8})
    got = np.concatenate(out[ids["sink"]]).reshape(-1, H, W)
    net.close()
    np.testing.assert_array_equal(got, MP.pipeline(f))


def test_streamed_motion_detector(P):
    from paper_1611_03226_b300.stream import stream
    T, H, W = 24, 1080, 1920
    f = synth.motion(n_frames=T).frames()[:T]
    tiles = (-(-H // 16)) * (-(-W // 16))
    net, ids = EN.motion_fused(P.Net, H, W, 6, tiles * 6)
    out, _ = stream(net, {ids["src"]: batches(f, 4, 1, 3)}, {ids["rec"]: tiles * 4, ids["cnt"]: 8})
    rec = np.concatenate(out[ids["rec"]]).view(MD.RECORD_DTYPE)
    cnt = np.concatenate(out[ids["cnt"]]).view(np.uint32)
    net.close()
    want_r, want_c = [], []
    prev = np.zeros((H, W), np.uint8)
    for t in range(T):
        r = MD.detect(f[t], prev)
        want_r.append(r)
        want_c.append(len(r))
        prev = f[t]
    np.testing.assert_array_equal(cnt, np.array(want_c, np.uint32))
    np.testing.assert_array_equal(rec, np.concatenate(want_r))


# ---- the native runner (df_stream): host actors as C++ threads ----

def oracle_dpd(w, masks, x):
    n = len(masks)
    onet, oi = ON.dpd_fused(w.h, w.orders, w.block_len, w.delay, n + w.delay)
    onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks))
    onet.push(oi["data"], ON.as_tokens_blocks(x))
    onet.run(-1)
    return np.array(onet.pop(oi["sink"]))


@pytest.mark.parametrize("flags", ["per_phase", "graph", "persistent"])
def test_native_stream_predistorter(P, flags):
    from paper_1611_03226_b300 import _lib as L
    fl = {"per_phase": 0, "graph": L.DF_RUN_GRAPH, "persistent": L.DF_RUN_PERSISTENT}[flags]
    w = synth.dpd_tiny()
    n, Lb = 40, w.block_len
    x, masks = np.ascontiguousarray(w.blocks(0, n)), np.ascontiguousarray(w.masks[:n])
    net, ids = EN.dpd_fused(P.Net, w.h, w.orders, Lb, w.delay, w.capacity)
    y = np.zeros((n + 5, Lb), np.complex64)
    popped, steps = net.stream({ids["ctrl"]: (masks, 1), ids["data"]: (x, 2)}, {ids["sink"]: (y, 3)}, fl)
    net.close()
    assert popped[ids["sink"]] == n and steps >= n // w.capacity
    want = oracle_dpd(w, masks, x)
    for i in range(n):
        assert np.linalg.norm(y[i] - want[i]) <= 1e-5 * max(np.linalg.norm(want[i]), 1e-30)
    assert not y[n:].any()


@pytest.mark.parametrize("cap,batch", [(9, 8), ("eq1", 4)])
def test_native_stream_paper_pipeline(P, cap, batch):
    """Ring buffers of 9 frames, or the paper's own Eq. 1 buffers (8-frame double
    buffers, a 13-slot Fig. 2 delay buffer) fed one window of 4 frames at a time."""
    T, H, W, rate = 64, 240, 320, 4
    f = synth.motion(n_frames=T, height=H, width=W).frames()
    net, ids = EN.motion_paper(P.Net, H, W, cap, rate)
    out = np.zeros_like(f)
    popped, _ = net.stream({ids["src"]: (f, batch)}, {ids["sink"]: (out, 8)})
    net.close()
    assert popped[ids["sink"]] == T
    np.testing.assert_array_equal(out, MP.pipeline(f))


def test_native_stream_motion_detector_from_device_memory(P):
    """Frames fed from device memory; two drains (records, per-frame counts)."""
    import torch
    T, H, W = 24, 1080, 1920
    f = synth.motion(n_frames=T).frames()[:T]
    tiles = (-(-H // 16)) * (-(-W // 16))
    net, ids = EN.motion_fused(P.Net, H, W, 6, tiles * 6)
    fd = torch.from_numpy(f).cuda()
    rec = np.zeros(tiles * T, MD.RECORD_DTYPE)
    cnt = np.zeros(T, np.uint32)
    popped, _ = net.stream({ids["src"]: (fd, 3)}, {ids["rec"]: (rec, tiles * 4), ids["cnt"]: (cnt, 8)})
    net.close()
    want_r, want_c, prev = [], [], np.zeros((H, W), np.uint8)
    for t in range(T):
        r = MD.detect(f[t], prev)
        want_r.append(r)
        want_c.append(len(r))
        prev = f[t]
    want_r = np.concatenate(want_r)
    assert popped[ids["cnt"]] == T and popped[ids["rec"]] == len(want_r)
    np.testing.assert_array_equal(cnt, np.array(want_c, np.uint32))
    np.testing.assert_array_equal(rec[:len(want_r)], want_r)


def test_native_stream_reports_a_stalled_network(P):
    """A sink nobody drains fills up: nothing can move, the run stops with
    DF_EDEADLOCK after the idle limit, and the network stays usable."""
    from paper_1611_03226_b300 import _lib as L
    net = P.Net()
    src, cp, s0, s1 = net.add_source(), net.add_copy(), net.add_sink(), net.add_sink()
    net.connect(src, 0, cp, 0, 16, 1, 4)
    net.connect(cp, 0, s0, 0, 16, 1, 4)
    net.connect(cp, 1, s1, 0, 16, 1, 2)           # not drained
    net.finalize()
    data = np.arange(16 * 20, dtype=np.uint8)
    out = np.zeros(16 * 20, np.uint8)
    with pytest.raises(L.DfError) as e:
        net.stream({src: (data, 2)}, {s0: (out, 4)}, idle_limit_s=0.3)
    assert e.value.status == L.DF_EDEADLOCK
    got = net.pop(s1)
    np.testing.assert_array_equal(got, data[:32])
    net.close()
