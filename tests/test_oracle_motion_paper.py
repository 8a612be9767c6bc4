"""Pins of the oracle for the paper's motion pipeline (Sec. 4.1: Gauss 5x5 with
the two top and bottom rows unfiltered, threshold of consecutive filtered
frames, 5-pixel median), against closed forms, scipy and brute force."""
import numpy as np
import pytest
from scipy import ndimage

import synth
from oracle import motion_paper as MP
from oracle import nets as ON

W5 = np.array(MP.GAUSS_ROW, np.int64)


def test_gauss_constant_frame_is_unchanged():
    for v in (0, 1, 77, 254, 255):
        f = np.full((12, 9), v, np.uint8)
        assert np.array_equal(MP.gauss5(f), f)


def test_gauss_skips_two_rows_top_and_bottom():
    f = synth.uniform_frames(1, 11, 16)[0]
    g = MP.gauss5(f)
    for y in (0, 1, 9, 10):
        assert np.array_equal(g[y], f[y])
    assert not np.array_equal(g[2:9], f[2:9])


def test_gauss_interior_equals_scipy_correlation_with_clamped_columns():
    f = synth.uniform_frames(1, 30, 41)[0]
    k = np.outer(W5, W5)
    assert k.sum() == 256
    ref = ndimage.correlate(f.astype(np.int64), k, mode="nearest")
    want = ((ref + 128) // 256).astype(np.uint8)
    g = MP.gauss5(f)
    # rows 2 .. H-3 are filtered; their vertical taps stay inside the frame, so only the
    # column clamp of mode "nearest" matters
    assert np.array_equal(g[2:-2], want[2:-2])


def test_gauss_impulse_response_closed_form():
    f = np.zeros((15, 15), np.uint8)
    f[7, 7] = 255
    g = MP.gauss5(f).astype(np.int64)
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            w = int(W5[dy + 2] * W5[dx + 2])
            assert g[7 + dy, 7 + dx] == (255 * w + 128) // 256
    mask = np.ones_like(g, bool)
    mask[5:10, 5:10] = False
    assert not g[mask].any()


def test_thres_brute_force_all_byte_pairs():
    a = np.repeat(np.arange(256, dtype=np.uint8), 256).reshape(256, 256)
    b = a.T.copy()
    for t in (0, 20, 128, 255):
        m = MP.thres(a, b, t)
        for i in range(0, 256, 17):
            for j in range(0, 256, 13):
                assert m[i, j] == (255 if abs(int(a[i, j]) - int(b[i, j])) > t else 0)


def test_med5_equals_scipy_median_with_plus_footprint():
    f = synth.uniform_frames(1, 23, 37)[0]
    plus = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], bool)
    ref = ndimage.median_filter(f, footprint=plus, mode="nearest")
    m = MP.med5(f)
    assert np.array_equal(m[1:-1, 1:-1], ref[1:-1, 1:-1])
    assert np.array_equal(m[0], f[0]) and np.array_equal(m[-1], f[-1])
    assert np.array_equal(m[:, 0], f[:, 0]) and np.array_equal(m[:, -1], f[:, -1])


def test_med5_of_a_binary_map_is_a_majority_vote():
    rng = np.random.default_rng(5)
    b = (rng.random((20, 20)) < 0.5).astype(np.uint8) * 255
    m = MP.med5(b)
    for y in range(1, 19):
        for x in range(1, 19):
            votes = sum(int(b[y + dy, x + dx] > 0) for dy, dx in ((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)))
            assert m[y, x] == (255 if votes >= 3 else 0)


def test_pipeline_constant_frames_give_no_motion_after_the_first():
    f = np.full((6, 16, 24), 90, np.uint8)
    out = MP.pipeline(f, initial=MP.gauss5(f[0]))
    assert not out.any()
    # against the zero initial token frame 0 is all motion (|90 - 0| > 20) except the median's
    # border copy, which is motion too
    assert (MP.pipeline(f[:1])[0] == 255).all()


def test_pipeline_isolated_noise_pixel_is_removed_by_the_median():
    a = np.full((16, 16), 100, np.uint8)
    b = a.copy()
    b[8, 8] = 255                    # after the Gaussian: a 5x5 blob, thresholded to its core
    g = MP.gauss5(b)
    m = MP.thres(g, MP.gauss5(a))
    core = m[6:11, 6:11] > 0
    assert core[2, 2] and core.sum() >= 1
    single = np.zeros((9, 9), np.uint8)
    single[4, 4] = 255
    assert not MP.med5(single).any()


def test_network_equals_direct_composition_and_is_scheduler_independent():
    f = synth.motion(n_frames=12, height=20, width=32).frames()
    want = MP.pipeline(f)
    for rate, cap in ((1, 3), (4, 9), (3, 7)):
        net, ids = ON.motion_paper(20, 32, cap, rate)
        n_whole = (len(f) // rate) * rate
        got = []
        for i in range(0, n_whole, rate):
            net.push(ids["src"], list(f[i:i + rate]))
            net.run(-1)
            got += net.pop(ids["sink"])
        assert np.array_equal(np.array(got), want[:n_whole])
    # random firing order reaches the same output stream
    net, ids = ON.motion_paper(20, 32, 16, 4)
    net.push(ids["src"], list(f[:12]))
    net.run_random(np.random.default_rng(1))
    assert np.array_equal(np.array(net.pop(ids["sink"])), want)


@pytest.mark.parametrize("mutant", ["weights", "rows", "threshold", "median"])
def test_pins_catch_planted_mistakes(mutant, monkeypatch):
    """Each plausible slip in the oracle breaks at least one pin above."""
    if mutant == "weights":
        monkeypatch.setattr(MP, "GAUSS_ROW", (1, 4, 6, 4, 2))
        with pytest.raises(AssertionError):
            test_gauss_interior_equals_scipy_correlation_with_clamped_columns()
    elif mutant == "rows":
        # filters row 1 and row H-2 as well (one skipped row instead of two)
        orig = MP.gauss5
        monkeypatch.setattr(MP, "gauss5", lambda fr: orig(np.pad(fr, 1, mode="edge"))[1:-1, 1:-1])
        with pytest.raises(AssertionError):
            test_gauss_skips_two_rows_top_and_bottom()
    elif mutant == "threshold":
        monkeypatch.setattr(MP, "thres", lambda c, p, t=20: np.where(
            np.abs(c.astype(int) - p.astype(int)) >= t, 255, 0).astype(np.uint8))
        with pytest.raises(AssertionError):
            test_thres_brute_force_all_byte_pairs()
    else:
        def med4(m):
            out = m.copy()
            four = np.stack([m[:-2, 1:-1], m[2:, 1:-1], m[1:-1, :-2], m[1:-1, 2:], m[1:-1, 1:-1] * 0])
            out[1:-1, 1:-1] = np.sort(four, axis=0)[2]
            return out
        monkeypatch.setattr(MP, "med5", med4)
        with pytest.raises(AssertionError):
            test_med5_equals_scipy_median_with_plus_footprint()
