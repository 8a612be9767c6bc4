"""Bit-exact parity of the fused motion detector (CUDA) with the integer oracle."""
import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import motion as MD
from oracle import nets as ON

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Net():
    from paper_1611_03226_b300 import Net
    return Net


def stream_both(Net, frames, cap, chunk, rec_capacity=None, separate=False, prev_init=None, flags=0,
                t=25):
    T, H, W = frames.shape
    onet, oi = ON.motion_fused(H, W, cap, rec_capacity, t=t, prev_init=prev_init)
    enet, ei = EN.motion_fused(Net, H, W, cap, rec_capacity, t=t, prev_init=prev_init,
                               separate_prev_source=separate)
    ro, co, re_, ce = [], [], [], []
    i, idle, n_step = 0, 0, 0
    cycle = flags if isinstance(flags, (list, tuple)) else [flags]
    while True:
        free = min(onet.channels[oi["ch_cur"]].free, onet.channels[oi["ch_prev"]].free)
        k = min(chunk, T - i, free)
        if k > 0:
            onet.push(oi["src"], list(frames[i:i + k]))
            enet.push(ei["src"], np.ascontiguousarray(frames[i:i + k]))
            if separate:
                enet.push(ei["src_prev"], np.ascontiguousarray(frames[i:i + k]))
            i += k
        fo, fe = onet.run(1), enet.run(1, cycle[n_step % len(cycle)])
        n_step += 1
        assert fo == fe
        for key in ("ch_cur", "ch_prev", "ch_rec", "ch_cnt"):
            assert onet.counters(oi[key]) == enet.counters(ei[key]), key
        ro += onet.pop(oi["rec"])
        co += onet.pop(oi["cnt"])
        re_.append(enet.pop(ei["rec"], dtype=MD.RECORD_DTYPE))
        ce.append(enet.pop(ei["cnt"], dtype=np.uint32))
        if i >= T and fo == 0:
            idle += 1
            if idle > 1:
                break
    enet.close()
    return (ON.records_of(ro), np.array([int(c[0]) for c in co], np.uint32),
            np.concatenate(re_), np.concatenate(ce))


@pytest.mark.parametrize("H,W,T,cap,chunk", [
    (72, 96, 9, 3, 2),          # ragged strip (72 = 4*16 + 8), 3 words per row
    (16, 32, 5, 2, 1),          # one strip, one word
    (37, 64, 6, 4, 3),
    (1080, 1920, 6, 4, 4),      # full-size frames
    (100, 544, 23, 11, 9),      # two bands (the second partial), units across the ring's end, odd chunks
    (50, 1024, 17, 17, 17),     # three bands, 8-frame units from the first frame on
    (1080, 1920, 19, 10, 10),   # full-size frames, 8-frame units across the ring's end
])
def test_motion_parity(Net, H, W, T, cap, chunk):
    w = synth.motion(n_frames=T, height=H, width=W)
    f = w.frames()
    ro, co, re_, ce = stream_both(Net, f, cap, chunk)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)
    assert ce.sum() == len(re_)


@pytest.mark.parametrize("t", [0, 1, 126, 127, 128, 129, 200, 254, 255])
@pytest.mark.parametrize("separate,flags", [(False, 0), (True, 0), (False, "persistent")])
def test_motion_thresholds(Net, t, separate, flags):
    """Every threshold class of the bytewise compare (below, at and above 128),
    on frames whose pixel differences span 0..255, through the shared-row
    kernel, the separate-previous-frame kernel and the persistent kernel."""
    from paper_1611_03226_b300 import _lib as L
    f = synth.blocky_frames(10, 40, 96) if t >= 120 else synth.uniform_frames(10, 40, 96)
    fl = L.DF_RUN_PERSISTENT if flags == "persistent" else 0
    ro, co, re_, ce = stream_both(Net, f, 9, 9, separate=separate, flags=fl, t=t)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)
    if t <= 127:
        assert len(re_) > 0


def test_motion_without_dedup(Net):
    """Previous frames from a channel of their own (no reuse of the current stream)."""
    w = synth.motion(n_frames=5, height=48, width=64)
    f = w.frames()
    ro, co, re_, ce = stream_both(Net, f, 3, 2, separate=True)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)


def test_constant_frames_and_initial_frame(Net):
    f = np.full((5, 40, 64), 99, np.uint8)
    ro, co, re_, ce = stream_both(Net, f, 3, 2, prev_init=f[0])
    assert len(re_) == 0 and list(ce) == [0] * 5


def test_record_fifo_backpressure(Net):
    """Record capacity of one frame's worth: the detector fires one frame per pop."""
    f = np.zeros((4, 32, 32), np.uint8)
    f[1::2] = 200
    ro, co, re_, ce = stream_both(Net, f, 4, 4, rec_capacity=4)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)


@pytest.mark.slow
def test_motion_full_workload(Net):
    """300 frames 1080p pushed whole, one run (the bench launch configuration):
    every count token and every record against the oracle."""
    w = synth.motion()
    f = w.frames()
    T, H, W = f.shape
    enet, ei = EN.motion_fused(Net, H, W, T + 1)
    enet.push(ei["src"], f)
    assert enet.run(-1) == T
    rec = enet.pop(ei["rec"], dtype=MD.RECORD_DTYPE)
    cnt = enet.pop(ei["cnt"], dtype=np.uint32)
    enet.close()
    want_c, want_r = [], []
    prev = np.zeros((H, W), np.uint8)
    for t in range(T):
        r = MD.detect(f[t], prev)
        want_c.append(len(r))
        want_r.append(r)
        prev = f[t]
    np.testing.assert_array_equal(cnt, np.array(want_c, np.uint32))
    np.testing.assert_array_equal(rec, np.concatenate(want_r))


@pytest.mark.parametrize("separate", [False, True])
def test_motion_persistent_mode(Net, separate):
    from paper_1611_03226_b300 import _lib as L
    w = synth.motion(n_frames=7, height=72, width=96)
    f = w.frames()
    ro, co, re_, ce = stream_both(Net, f, 3, 2, separate=separate, flags=L.DF_RUN_PERSISTENT)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)


@pytest.mark.parametrize("H,W", [(72, 96), (1080, 1920)])
def test_motion_launch_modes_alternate(Net, H, W):
    """Steps launched eagerly, from a graph and as the persistent kernel in
    turn (the TMA main kernel at these widths, the register-staged one inside
    the persistent kernel): every step's counters, records and count tokens
    equal the oracle's."""
    from paper_1611_03226_b300 import _lib as L
    w = synth.motion(n_frames=13, height=H, width=W)
    f = w.frames()
    modes = [0, L.DF_RUN_GRAPH, L.DF_RUN_PERSISTENT, L.DF_RUN_GRAPH, 0, L.DF_RUN_PERSISTENT | L.DF_RUN_GRAPH]
    ro, co, re_, ce = stream_both(Net, f, 4, 3, flags=modes)
    np.testing.assert_array_equal(ce, co)
    np.testing.assert_array_equal(re_, ro)
