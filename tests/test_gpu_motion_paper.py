"""Bit-exact parity of the paper's motion pipeline (Gauss -> Thres -> Med,
Sec. 4.1) through the engine with the integer oracle, step by step, with the
channel counters compared after every step."""
import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import motion_paper as MP
from oracle import nets as ON

pytestmark = pytest.mark.gpu

CHANNELS = ("ch_in", "ch_cur", "ch_prev", "ch_map", "ch_out")


@pytest.fixture(scope="module")
def Net():
    from paper_1611_03226_b300 import Net
    return Net


def stream_both(Net, frames, cap, rate, chunk, t=20, initial=None, flags=0):
    T, H, W = frames.shape
    onet, oi = ON.motion_paper(H, W, cap, rate, t, initial)
    enet, ei = EN.motion_paper(Net, H, W, cap, rate, t, initial)
    got, want = [], []
    i, idle = 0, 0
    while True:
        k = min(chunk, T - i, onet.channels[oi["ch_in"]].free)
        if k > 0:
            onet.push(oi["src"], list(frames[i:i + k]))
            enet.push(ei["src"], np.ascontiguousarray(frames[i:i + k]))
            i += k
        fo, fe = onet.run(1), enet.run(1, flags)
        assert fo == fe
        for key in CHANNELS:
            assert onet.counters(oi[key]) == enet.counters(ei[key]), key
        want += onet.pop(oi["sink"])
        got.append(enet.pop(ei["sink"], dtype=np.uint8))
        if i >= T and fo == 0:
            idle += 1
            if idle > 1:
                break
    enet.close()
    got = np.concatenate(got).reshape(-1, H, W)
    return got, np.array(want, np.uint8).reshape(-1, H, W)


@pytest.mark.parametrize("H,W,T,cap,rate,chunk", [
    (240, 320, 21, 9, 4, 8),     # the paper's frame size at rate 4; 20 of 21 frames fire
    (37, 48, 11, 5, 1, 2),       # ragged band (37 = 2*16 + 5), rate 1
    (18, 16, 9, 7, 3, 6),        # one 16-pixel column group, rate 3
    (5, 32, 6, 4, 1, 3),         # one filtered row
    (4, 16, 5, 4, 1, 2),         # no filtered rows
    (2, 16, 4, 3, 1, 1),         # median copies everything
])
def test_parity(Net, H, W, T, cap, rate, chunk):
    f = synth.motion(n_frames=T, height=H, width=W).frames() if H >= 16 else synth.uniform_frames(T, H, W)
    got, want = stream_both(Net, f, cap, rate, chunk)
    assert len(want) == (T // rate) * rate
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(want, MP.pipeline(f[:len(want)]))


@pytest.mark.parametrize("t", [0, 1, 128, 254, 255])
def test_thresholds_and_initial_frame(Net, t):
    f = synth.uniform_frames(8, 40, 64)
    init = synth.uniform_frames(1, 40, 64, seed=7)[0]
    got, want = stream_both(Net, f, 10, 2, 4, t=t, initial=init)
    np.testing.assert_array_equal(got, want)


def test_persistent_mode(Net):
    from paper_1611_03226_b300 import _lib as L
    f = synth.motion(n_frames=12, height=48, width=64).frames()
    got, want = stream_both(Net, f, 9, 4, 8, flags=L.DF_RUN_PERSISTENT)
    np.testing.assert_array_equal(got, want)


def test_whole_video_in_one_run(Net):
    """All frames pushed at once and run to quiescence (the bench configuration)."""
    T, H, W, rate = 64, 240, 320, 4
    f = synth.motion(n_frames=T, height=H, width=W).frames()
    net, ids = EN.motion_paper(Net, H, W, T + 1, rate)
    net.push(ids["src"], f)
    assert net.run(-1) == 3 * (T // rate)
    got = net.pop(ids["sink"], dtype=np.uint8).reshape(-1, H, W)
    net.close()
    np.testing.assert_array_equal(got, MP.pipeline(f))


@pytest.mark.parametrize("kind", ["gauss", "med"])
@pytest.mark.parametrize("H,W,n_out", [
    (240, 320, 2), (19, 48, 2), (3, 16, 2),
    (37, 1040, 3),     # wider than 1024: 16-row bands, 65 units a row, a ragged last band, a third output
    (20, 2048, 1),     # the widest frame: 2048 units a band, 8 a thread
])
def test_single_actor_on_gray_frames(Net, kind, H, W, n_out):
    """Gauss or Med alone on arbitrary 8-bit frames (the median's general path,
    not only the 0/255 maps the pipeline feeds it), one to three output channels."""
    T, rate = 6, 2
    f = synth.uniform_frames(T, H, W, seed=11) if H < 16 else synth.motion(n_frames=T, height=H, width=W).frames()
    if kind == "med":
        f = synth.uniform_frames(T, H, W, seed=12)
    net = Net()
    fb = H * W
    src = net.add_source()
    act = net.add_gauss5(W, H) if kind == "gauss" else net.add_med5(W, H)
    sinks = [net.add_sink() for _ in range(n_out)]
    net.connect(src, 0, act, 0, fb, rate, T)
    for p, s in enumerate(sinks):
        net.connect(act, p, s, 0, fb, rate, T)
    net.finalize()
    net.push(src, f)
    assert net.run(-1) == T // rate
    want = np.stack([(MP.gauss5 if kind == "gauss" else MP.med5)(x) for x in f])
    for s in sinks:
        np.testing.assert_array_equal(net.pop(s, dtype=np.uint8).reshape(T, H, W), want)
    net.close()


@pytest.mark.parametrize("wiring", ["two_sources", "delay_on_first_input", "one_source"])
def test_thres_input_wirings(Net, wiring):
    """Thres reads its previous frames from the current input only when the second input
    is the first one's stream one token later (one broadcast writer, delay on input 1);
    the other wirings take every frame from its own channel."""
    T, H, W, rate, t = 12, 24, 48, 2, 20
    a = synth.uniform_frames(T, H, W, seed=21)
    b = synth.uniform_frames(T, H, W, seed=22)
    init = synth.uniform_frames(1, H, W, seed=23)[0]
    fb = H * W
    net = Net()
    s0 = net.add_source()
    s1 = net.add_source() if wiring == "two_sources" else s0
    th, snk = net.add_thres(W, H, t), net.add_sink()
    d0, d1 = (1, 0) if wiring == "delay_on_first_input" else (0, 1 if wiring == "one_source" else 0)
    net.connect(s0, 0, th, 0, fb, rate, T + 1, d0, init if d0 else None)
    net.connect(s1, 1 if s1 == s0 else 0, th, 1, fb, rate, T + 1, d1, init if d1 else None)
    net.connect(th, 0, snk, 0, fb, rate, T + 1)
    net.finalize()
    net.push(s0, a)
    if wiring == "two_sources":
        net.push(s1, b)
    net.run(-1)
    got = net.pop(snk, dtype=np.uint8).reshape(-1, H, W)
    net.close()
    if wiring == "two_sources":
        first, second = a, b
    elif wiring == "delay_on_first_input":
        first, second = np.concatenate([init[None], a]), a
    else:
        first, second = a, np.concatenate([init[None], a])
    n = min(len(first), len(second)) // rate * rate
    assert len(got) == n
    np.testing.assert_array_equal(got, np.stack([MP.thres(first[i], second[i], t) for i in range(n)]))


@pytest.mark.parametrize("binary_init", [True, False])
def test_med_after_thres_with_initial_frame(Net, binary_init):
    """Med reading Thres's 0/255 maps takes the bitwise-majority path without a
    per-band check; an initial frame on its input channel that is not 0/255
    keeps the general median (the engine decides this when it is built)."""
    T, H, W, rate, t = 8, 24, 48, 2, 20
    f = synth.uniform_frames(T, H, W, seed=31)
    init = synth.uniform_frames(1, H, W, seed=32)[0]
    if binary_init:
        init = np.where(init > 127, 255, 0).astype(np.uint8)
    fb = H * W
    net = Net()
    src, th, med, snk = net.add_source(), net.add_thres(W, H, t), net.add_med5(W, H), net.add_sink()
    net.connect(src, 0, th, 0, fb, rate, T + 1)
    net.connect(src, 1, th, 1, fb, rate, T + 1, 1)
    net.connect(th, 0, med, 0, fb, rate, T + 2, 1, init)
    net.connect(med, 0, snk, 0, fb, rate, T + 2)
    net.finalize()
    net.push(src, f)
    net.run(-1)
    got = net.pop(snk, dtype=np.uint8).reshape(-1, H, W)
    net.close()
    prev = np.concatenate([np.zeros((1, H, W), np.uint8), f[:-1]])
    maps = np.stack([MP.thres(f[i], prev[i], t) for i in range(T)])
    want = np.stack([MP.med5(x) for x in np.concatenate([init[None], maps])])
    n = len(got)
    assert n >= T - rate
    np.testing.assert_array_equal(got, want[:n])
