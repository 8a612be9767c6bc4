"""Pins for the motion-detection oracle (exact integers)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import motion as MD
from oracle import nets

import synth


def run_all(net, ids, frames, chunk=2):
    recs, cnts = [], []
    i = 0
    while True:
        k = min(chunk, len(frames) - i, net.channels[ids["ch_cur"]].free,
                net.channels[ids["ch_prev"]].free)
        if k > 0:
            net.push(ids["src"], list(frames[i:i + k]))
            i += k
        fired = net.run(1)
        recs += net.pop(ids["rec"])
        cnts += net.pop(ids["cnt"])
        if i >= len(frames) and fired == 0:
            break
    return nets.records_of(recs), np.array([int(c[0]) for c in cnts], np.int64)


def test_constant_frames_no_motion_p8():
    H, W = 40, 72
    f = np.full((6, H, W), 77, np.uint8)
    net, ids = nets.motion_fused(H, W, capacity=3, prev_init=f[0])
    rec, cnt = run_all(net, ids, f)
    assert len(rec) == 0 and list(cnt) == [0] * 6
    # with the default zero initial frame only frame 0 shows motion (every pixel > 25)
    net, ids = nets.motion_fused(H, W, capacity=3)
    rec, cnt = run_all(net, ids, f)
    assert cnt[0] == 3 * 5 and list(cnt[1:]) == [0] * 5


def test_threshold_is_strict():
    d = np.array([[24, 25, 26, 255]], np.uint8)
    np.testing.assert_array_equal(MD.threshold(d, 25), [[0, 0, 1, 1]])
    a = np.array([[0, 10, 200]], np.uint8)
    b = np.array([[255, 36, 0]], np.uint8)
    np.testing.assert_array_equal(MD.absdiff(a, b), [[255, 26, 200]])


def test_morphology_matches_scipy_p10():
    rng = np.random.default_rng(3)
    s = np.ones((3, 3), bool)
    for p in (0.3, 0.6, 0.85):
        b = (rng.random((37, 53)) < p).astype(np.uint8)
        e = ndimage.binary_erosion(b, s, border_value=1).astype(np.uint8)
        dl = ndimage.binary_dilation(b, s, border_value=0).astype(np.uint8)
        np.testing.assert_array_equal(MD.erode3x3(b), e)
        np.testing.assert_array_equal(MD.dilate3x3(b), dl)


def test_translated_rectangle_closed_form_p9():
    """Flat background, one rectangle moving right by dx (noise off, contrast 80):
    the motion mask is the two dx-wide strips the rectangle enters and leaves,
    which a 3x3 opening leaves unchanged when dx >= 3 and the strips are >= 3 tall."""
    H, W, rw, rh, x0, y0, dx = 70, 100, 30, 21, 5, 9, 7
    fr = synth.flat_with_rect(H, W, 2, rw, rh, x0, y0, dx)
    o = MD.dilate3x3(MD.erode3x3(MD.threshold(MD.absdiff(fr[1], fr[0]))))
    want = np.zeros((H, W), np.uint8)
    want[y0:y0 + rh, x0:x0 + dx] = 1                    # uncovered background
    want[y0:y0 + rh, x0 + rw:x0 + rw + dx] = 1          # newly covered
    np.testing.assert_array_equal(o, want)
    cnt = MD.tile_counts(o)
    assert cnt.shape == (5, 7)                          # ceil(70/16), ceil(100/16)

    def area(ty, tx):                                   # strip-tile intersection area
        ys = max(0, min(16 * ty + 16, y0 + rh) - max(16 * ty, y0))
        xs = sum(max(0, min(16 * tx + 16, a + dx) - max(16 * tx, a)) for a in (x0, x0 + rw))
        return ys * xs

    for ty in range(5):
        for tx in range(7):
            assert cnt[ty, tx] == area(ty, tx)
    assert int(cnt.sum()) == 2 * dx * rh
    rec = MD.tile_records(cnt)
    want = [(16 * tx, 16 * ty, area(ty, tx)) for ty in range(5) for tx in range(7) if area(ty, tx)]
    assert [(int(r["x"]), int(r["y"]), int(r["count"])) for r in rec] == want   # raster order


def test_ragged_last_tile_row():
    H, W = 1080, 64                   # 1080 = 67*16 + 8
    o = np.ones((H, W), np.uint8)
    c = MD.tile_counts(o)
    assert c.shape == (68, 4) and np.all(c[:67] == 256) and np.all(c[67] == 128)


def test_literal_network_equals_fused():
    w = synth.motion(n_frames=7, height=72, width=96)
    f = w.frames()
    a, ai = nets.motion_literal(72, 96, capacity=2)
    b, bi = nets.motion_fused(72, 96, capacity=3)
    ra, ca = run_all(a, ai, f, chunk=1)
    rb, cb = run_all(b, bi, f, chunk=3)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(ra, rb)
    assert ca.sum() == len(ra) and ca.sum() > 0


def test_variable_rate_output_blocks_when_full():
    """With record capacity below r_max + something the detector waits for the sink."""
    H, W = 32, 32
    f = np.zeros((3, H, W), np.uint8)
    f[1] = 200
    n_tiles = 4
    net, ids = nets.motion_fused(H, W, capacity=4, rec_capacity=n_tiles)
    net.push(ids["src"], list(f))
    net.run(-1)
    assert net.counters(ids["ch_cnt"])[0] == 2        # frames 0, 1 fire; frame 1 fills the FIFO
    assert len(net.pop(ids["rec"])) == 4
    net.run(-1)
    assert net.counters(ids["ch_cnt"])[0] == 3
