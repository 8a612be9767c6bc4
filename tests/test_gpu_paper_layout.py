"""The paper's channel layout (Sec. 3.2: Eq. 1 sizes, the Fig. 2 access pattern)
on the engine.  Buffer sizes of the motion pipeline against Table 1; the raw
slots of double and delay buffers, after every step, against the oracle's
sequential buffer models replayed with the windows the counters show (so the
Fig. 2 pattern, the slot 3r -> 0 copy included, is checked byte for byte);
and parity of the networks built with it: the paper's motion pipeline, copy
chains whose delay channels are written by device actors, the fused and the
expanded predistorter."""
import json
import os

import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import actors as A
from oracle import dpd as D
from oracle import motion_paper as MP
from oracle import nets as ON
from oracle import paper_layout as PL
from oracle.network import Network, Sink, Source

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MOTION_CH = ("ch_in", "ch_cur", "ch_prev", "ch_map", "ch_out")


@pytest.fixture(scope="module")
def P():
    import paper_1611_03226_b300 as P
    return P


def flag(P, mode):
    from paper_1611_03226_b300 import _lib as L
    return {"per_phase": 0, "graph": L.DF_RUN_GRAPH, "persistent": L.DF_RUN_PERSISTENT}[mode]


class SlotModel:
    """The oracle's buffer model of one channel, advanced to the windows its
    counters show; `tokens` are the tokens written after the initial one."""

    def __init__(self, r, delay_token=None):
        self.r = r
        self.buf = PL.TripleBuffer(r, delay_token) if delay_token is not None else PL.DoubleBuffer(r)

    def check(self, net, ch, tokens):
        produced, consumed, _ = net.counters(ch)
        r = self.r
        while self.buf.nw * r < produced:
            k = self.buf.nw
            self.buf.write(list(tokens[k * r:(k + 1) * r]))
        while self.buf.nr * r < consumed:
            self.buf.read()
        raw = net.peek_slots(ch)
        assert len(raw) == len(self.buf.slots)
        for s, t in enumerate(self.buf.slots):
            if t is not None:
                np.testing.assert_array_equal(raw[s], np.ascontiguousarray(t).reshape(-1).view(np.uint8),
                                              err_msg=f"slot {s}")


def test_table1_buffer_memory(P):
    """Sec. 4.1 with 320x240 frames (76 800-byte tokens) at rate 4: four double
    buffers of 8 slots and one delay buffer of 13, 45 slots = 3.456 MB, Table 1's
    3.46 MB (Prop., Heterog.); at rate 1, 12 slots."""
    g = json.load(open(os.path.join(GOLD, "table1_buffer_memory.json")))
    for rate in (g["motion_gpu_rate"], 1):
        net, ids = EN.motion_paper(P.Net, 240, 320, "eq1", rate)
        info = [net.channel_info(ids[k]) for k in MOTION_CH]
        assert [i["layout"] for i in info] == ["eq1"] * 5
        assert [i["capacity"] for i in info] == [2 * rate, 2 * rate, 3 * rate, 2 * rate, 2 * rate]
        assert [i["slots"] for i in info] == [2 * rate, 2 * rate, 3 * rate + 1, 2 * rate, 2 * rate]
        total = sum(i["buffer_bytes"] for i in info)
        if rate == g["motion_gpu_rate"]:
            assert total == 3456000 and round(total / 1e6, 2) == g["prop_heterog_MB"]
        else:
            assert total == 12 * 76800
        net.close()
    # a ring channel reports its own capacity as its size
    net = P.Net()
    a, b = net.add_source(), net.add_sink()
    c = net.connect(a, 0, b, 0, 16, 2, 7)
    assert net.channel_info(c) == {"capacity": 7, "slots": 7, "buffer_bytes": 112, "token_bytes": 16,
                                   "rate": 2, "initial_tokens": 0, "layout": "ring"}
    net.close()


def test_eq1_rejects_what_the_paper_does_not_define(P):
    from paper_1611_03226_b300 import _lib as L
    net = P.Net()
    a, b = net.add_source(), net.add_copy()
    with pytest.raises(L.DfError) as e:
        net.connect(a, 0, b, 0, 8, 2, "eq1", 2)                 # two delay tokens
    assert e.value.status == L.DF_EINVAL
    md = net.add_md(64, 32)
    s = net.add_sink()
    with pytest.raises(L.DfError) as e:
        net.connect(md, 1, s, 0, 4, 1, "eq1")                  # written by the motion detector
    assert e.value.status == L.DF_EINVAL
    net.close()


@pytest.mark.parametrize("H,W,T,rate,chunk", [
    (240, 320, 21, 4, 8),       # the paper's configuration: 8-frame double buffers, 13-slot delay buffer
    (37, 48, 13, 1, 2),         # rate 1: the delay buffer has 4 slots and wraps every 3 tokens
    (18, 16, 14, 3, 6),
])
@pytest.mark.parametrize("mode", ["per_phase", "graph", "persistent"])
def test_motion_pipeline_in_eq1_layout(P, H, W, T, rate, chunk, mode):
    f = synth.motion(n_frames=T, height=H, width=W).frames()
    g = np.stack([MP.gauss5(x) for x in f])
    onet, oi = ON.motion_paper(H, W, "eq1", rate)
    enet, ei = EN.motion_paper(P.Net, H, W, "eq1", rate)
    models = {"ch_in": (SlotModel(rate), f), "ch_cur": (SlotModel(rate), g),
              "ch_prev": (SlotModel(rate, np.zeros((H, W), np.uint8)), g)}
    got, want = [], []
    i, idle, spills = 0, 0, 0
    T_whole = T // rate * rate              # the source writes whole windows of r frames
    while True:
        k = min(chunk, T_whole - i, onet.channels[oi["ch_in"]].free)
        k -= k % rate
        if k > 0:
            onet.push(oi["src"], list(f[i:i + k]))
            enet.push(ei["src"], np.ascontiguousarray(f[i:i + k]))
            i += k
        fo, fe = onet.run(1), enet.run(1, flag(P, mode))
        assert fo == fe
        for key in MOTION_CH:
            assert onet.counters(oi[key]) == enet.counters(ei[key]), key
        for key, (m, toks) in models.items():
            m.check(enet, ei[key], toks)
        spills = models["ch_prev"][0].buf.nw // 3     # writes that filled slot 3r
        want += onet.pop(oi["sink"])
        got.append(enet.pop(ei["sink"], dtype=np.uint8))
        if i >= T_whole and fo == 0:
            idle += 1
            if idle > 1:
                break
    enet.close()
    got = np.concatenate(got).reshape(-1, H, W)
    assert len(got) == T_whole
    np.testing.assert_array_equal(got, np.array(want, np.uint8).reshape(-1, H, W))
    np.testing.assert_array_equal(got, MP.pipeline(f[:len(got)]))
    assert spills >= 1                      # the slot 3r -> 0 copy was exercised


@pytest.mark.parametrize("mode", ["per_phase", "persistent"])
def test_copy_chain_with_device_written_delay_buffers(P, mode):
    """source -(r 2, 6 B, delay)-> copy -(r 3, 4 B, delay)-> copy -(r 1, 12 B, delay)-> sink,
    every channel in the paper's layout: the second and third delay buffers are
    written by device copy actors, the first by the host."""
    rates, sizes = [2, 3, 1], [6, 4, 12]
    inits = [np.arange(s, dtype=np.uint8) + 100 + 10 * k for k, s in enumerate(sizes)]
    onet, enet = Network(), P.Net()
    o_prev, e_prev = onet.add_actor(Source()), enet.add_source()
    src_o, src_e = o_prev, e_prev
    chans = []
    for k in range(3):
        last = k == 2
        od = onet.add_actor(Sink() if last else A.Copy())
        ed = enet.add_sink() if last else enet.add_copy()
        chans.append((onet.connect(o_prev, 0, od, 0, rates[k], "eq1", [inits[k]], sizes[k]),
                      enet.connect(e_prev, 0, ed, 0, sizes[k], rates[k], "eq1", 1, inits[k])))
        o_prev, e_prev = od, ed
    onet.finalize()
    enet.finalize()
    # bytes written into channel k after its initial token
    rng = np.random.default_rng(3)
    pushed = rng.integers(0, 256, 6 * 60, dtype=np.uint8)
    written = [pushed]
    for k in range(1, 3):
        written.append(np.concatenate([inits[k - 1], written[k - 1]]))
    toks = [w[:len(w) // sizes[k] * sizes[k]].reshape(-1, sizes[k]) for k, w in enumerate(written)]
    models = [SlotModel(rates[k], inits[k]) for k in range(3)]
    seq, got_o, got_e = 0, [], []
    for it in range(40):
        free = onet.channels[chans[0][0]].free
        n = min(int(rng.integers(0, 3)) * 2, free - free % 2, 60 - seq)   # whole windows of 2
        if n > 0:
            onet.push(src_o, list(toks[0][seq:seq + n]))
            enet.push(src_e, np.ascontiguousarray(toks[0][seq:seq + n]))
            seq += n
        assert onet.run(1) == enet.run(1, flag(P, mode))
        for k, (oc, ec) in enumerate(chans):
            assert onet.counters(oc) == enet.counters(ec)
            models[k].check(enet, ec, toks[k])
        m = int(rng.integers(0, 3))
        got_o += onet.pop(o_prev, m)
        got_e.append(enet.pop(e_prev, m))
    want = np.concatenate(got_o)
    np.testing.assert_array_equal(np.concatenate(got_e), want)
    assert len(want) >= 12 * 20
    assert all(m.buf.nw >= 3 for m in models)      # every delay buffer filled slot 3r at least once
    enet.close()


def dpd_nets(P, h, orders, L, caps, delays):
    """ctrl, data -> DPD -> sink on both sides, channel (capacity, delay) per edge."""
    blk = L * 8
    onet = Network()
    oc, od = onet.add_actor(Source()), onet.add_actor(Source())
    odp, osk = onet.add_actor(A.Dpd(h, orders, L)), onet.add_actor(Sink())
    zero = np.zeros(L, np.complex128)
    onet.connect(oc, 0, odp, 0, 1, caps[0], token_bytes=4)
    onet.connect(od, 0, odp, 1, 1, caps[1], [zero] * delays[1], token_bytes=blk)
    onet.connect(odp, 0, osk, 0, 1, caps[2], [zero] * delays[2], token_bytes=blk)
    onet.finalize()
    enet = P.Net()
    ec, ed = enet.add_source(), enet.add_source()
    edp, esk = enet.add_dpd(h, orders, L), enet.add_sink()
    enet.connect(ec, 0, edp, 0, 4, 1, caps[0])
    enet.connect(ed, 0, edp, 1, blk, 1, caps[1], delays[1])
    enet.connect(edp, 0, esk, 0, blk, 1, caps[2], delays[2])
    enet.finalize()
    return onet, enet, (oc, od, osk), (ec, ed, esk)


@pytest.mark.parametrize("delays", [(0, 1, 0), (0, 0, 1), (0, 1, 1)])
@pytest.mark.parametrize("mode", ["per_phase", "graph", "persistent"])
def test_fused_predistorter_in_eq1_layout(P, delays, mode):
    """Delay on the data edge (the host writes the Fig. 2 buffer) and on the output
    edge (the predistorter body writes it)."""
    rng = np.random.default_rng(7 + sum(delays))
    n, L, K, M = 14, 300, 4, 10
    orders = (1, 3, 5, 7)
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    masks = rng.integers(1, 1 << K, n).astype(np.uint32)
    onet, enet, (oc, od, osk), (ec, ed, esk) = dpd_nets(P, h, orders, L, ["eq1"] * 3, delays)
    data_model = SlotModel(1, np.zeros(L, np.complex64)) if delays[1] else SlotModel(1)
    yo, ye, i = [], [], 0
    for step in range(60):
        k = min(1, n - i, onet.channels[0].free, onet.channels[1].free)
        if k > 0:
            onet.push(oc, ON.as_tokens_ctrl(masks[i:i + k]))
            onet.push(od, ON.as_tokens_blocks(x[i:i + k]))
            enet.push(ec, np.ascontiguousarray(masks[i:i + k]))
            enet.push(ed, np.ascontiguousarray(x[i:i + k]))
            i += k
        fo, fe = onet.run(1), enet.run(1, flag(P, mode))
        assert fo == fe
        for c in range(3):
            assert onet.counters(c) == enet.counters(c)
        data_model.check(enet, 1, x)
        yo += onet.pop(osk, 1)
        ye.append(enet.pop(esk, 1, dtype=np.complex64))
        if i >= n and fo == 0 and not onet.channels[2].occupancy:
            break
    enet.close()
    yo = np.array(yo).reshape(-1, L)
    ye = np.concatenate(ye).reshape(-1, L)
    assert len(ye) == len(yo) == n + delays[2]     # the last delays[1] data blocks stay queued
    for b in range(len(yo)):
        if not np.any(yo[b]):
            np.testing.assert_array_equal(ye[b], 0)
        else:
            assert D.rel_l2(ye[b], yo[b]) <= 1e-5


@pytest.mark.parametrize("mode", ["per_phase", "persistent"])
def test_expanded_predistorter_in_eq1_layout(P, mode):
    """Poly -> FIR_k -> Adder with every channel an Eq. 1 buffer (branch double
    buffers of 2 blocks, a delay buffer of 4 slots on the data edge)."""
    rng = np.random.default_rng(11)
    n, L, K, M = 12, 256, 3, 6
    orders = (1, 3, 5)
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    masks = rng.integers(0, 1 << K, n).astype(np.uint32)
    onet, oi = ON.dpd_expanded(h, orders, L, 1, "eq1")
    enet, ei = EN.dpd_expanded(P.Net, h, orders, L, 1, "eq1")
    assert enet.channel_info(ei["ch_data"])["slots"] == 4
    yo, ye, i = [], [], 0
    for step in range(200):
        free = min(onet.channels[0].free, onet.channels[1].free, onet.channels[oi["ch_data"]].free)
        k = min(2, n - i, free)
        if k > 0:
            onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks[i:i + k]))
            onet.push(oi["data"], ON.as_tokens_blocks(x[i:i + k]))
            enet.push(ei["ctrl"], np.ascontiguousarray(masks[i:i + k]))
            enet.push(ei["data"], np.ascontiguousarray(x[i:i + k]))
            i += k
        fo, fe = onet.run(1), enet.run(1, flag(P, mode))
        assert fo == fe
        for c in range(len(onet.channels)):
            assert onet.counters(c) == enet.counters(c), (step, c)
        yo += onet.pop(oi["sink"])
        ye.append(enet.pop(ei["sink"], dtype=np.complex64))
        if i >= n and fo == 0:
            break
    enet.close()
    yo = np.array(yo).reshape(-1, L)
    ye = np.concatenate(ye).reshape(-1, L)
    assert len(ye) == n
    for b in range(n):
        assert D.rel_l2(ye[b], yo[b]) <= 1e-5


def test_streamed_paper_pipeline_in_eq1_layout(P):
    """The paper's heterogeneous setting: host source and sink threads around the
    GPU actors, every buffer sized by Eq. 1 (8-frame double buffers at rate 4)."""
    from paper_1611_03226_b300.stream import stream
    T, H, W, rate = 64, 240, 320, 4
    f = synth.motion(n_frames=T, height=H, width=W).frames()
    net, ids = EN.motion_paper(P.Net, H, W, "eq1", rate)
    out, _ = stream(net, {ids["src"]: [f[i:i + rate] for i in range(0, T, rate)]}, {ids["sink"]: 2 * rate})
    got = np.concatenate(out[ids["sink"]]).reshape(-1, H, W)
    net.close()
    np.testing.assert_array_equal(got, MP.pipeline(f))


def test_layout_and_runner_error_paths(P):
    from paper_1611_03226_b300 import _lib as L
    net, ids = EN.motion_paper(P.Net, 24, 32, "eq1", 2)
    f = synth.uniform_frames(6, 24, 32)
    with pytest.raises(L.DfError) as e:
        net.push(ids["src"], f[:3])                            # not a whole window of 2 frames
    assert e.value.status == L.DF_EINVAL
    assert net.counters(ids["ch_in"]) == (0, 0, 0)              # nothing written
    with pytest.raises(L.DfError) as e:
        net.peek_slots(ids["ch_prev"], 6, 2)                    # the delay buffer has 7 slots
    assert e.value.status == L.DF_EINVAL
    with pytest.raises(L.DfError) as e:
        net.channel_info(99)
    assert e.value.status == L.DF_EINVAL
    out = np.zeros_like(f)
    with pytest.raises(L.DfError) as e:
        net.stream({ids["src"]: (f, 0)}, {ids["sink"]: (out, 2)})          # batch 0
    assert e.value.status == L.DF_EINVAL
    with pytest.raises(L.DfError) as e:
        net.stream({ids["src"]: (f, 2)}, {ids["sink"]: (out, 2)}, L.DF_RUN_ASYNC)
    assert e.value.status == L.DF_EINVAL
    fs = (L.Feed * 1)()
    fs[0] = L.Feed(ids["sink"], f.ctypes.data, 6, 2)                     # a sink is no source
    assert L.lib.df_stream(net.h, fs, 1, None, 0, 0, 0, None) == L.DF_EINVAL
    # the network is still usable: the paper's layout streamed by the persistent kernel
    popped, _ = net.stream({ids["src"]: (f, 2)}, {ids["sink"]: (out, 2)}, L.DF_RUN_PERSISTENT)
    assert popped[ids["sink"]] == 6
    np.testing.assert_array_equal(out, MP.pipeline(f))
    net.close()


@pytest.mark.parametrize("rate", [1, 3])
def test_broadcast_push_into_eq1_delay_buffer(P, rate):
    """A source broadcasting into two Eq. 1 channels of Thres, the second with one
    delay token: the push fills the delay buffer by a device copy from the first
    channel and makes the slot 3r -> 0 copy itself; Thres takes its previous frames
    from its current input.  Raw slots follow Fig. 2 after every push and step."""
    H, W, T = 16, 32, 6 * rate
    f = synth.uniform_frames(T, H, W, seed=31)
    init = synth.uniform_frames(1, H, W, seed=32)[0]
    net = P.Net()
    src, th, snk = net.add_source(), net.add_thres(W, H, 20), net.add_sink()
    c0 = net.connect(src, 0, th, 0, H * W, rate, "eq1")
    c1 = net.connect(src, 1, th, 1, H * W, rate, "eq1", 1, init)
    net.connect(th, 0, snk, 0, H * W, rate, "eq1")
    net.finalize()
    models = [(SlotModel(rate), c0), (SlotModel(rate, init), c1)]
    got = []
    for i in range(0, T, rate):
        net.push(src, f[i:i + rate])
        for m, c in models:
            m.check(net, c, f)
        net.run(1)
        for m, c in models:
            m.check(net, c, f)
        got.append(net.pop(snk, dtype=np.uint8))
    net.close()
    got = np.concatenate(got).reshape(-1, H, W)
    prev = np.concatenate([init[None], f[:-1]])
    np.testing.assert_array_equal(got, np.stack([MP.thres(f[i], prev[i], 20) for i in range(T)]))
    assert models[1][0].buf.nw >= 3                 # the delay buffer filled slot 3r at least once
