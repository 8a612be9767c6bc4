"""The paper's own motion-detection pipeline, Sec. 4.1 (test infrastructure).

Five actors (Fig. 3; the figure is lost, its structure is taken from the
text): a source, Gauss, Thres, Med and a sink.  Gauss applies a 5x5 Gaussian
filter to every frame, leaving the two top and the two bottom pixel rows
unfiltered; Thres subtracts consecutive filtered frames (one of its two input
channels carries an initial token, a one-frame delay) and thresholds the
difference against a constant; Med applies a 5-pixel median filter to the
resulting motion map.  Frames are 8-bit grayscale, 320x240 in the paper.

The paper leaves the filter weights, the column border, the threshold
constant, the threshold's output values and the median's shape open.  This
oracle takes these readings:

* Gauss weights: the binomial row (1, 4, 6, 4, 1) in both directions, so the
  5x5 weight of (dy, dx) is w[dy] * w[dx] with a total of 256; the result is
  rounded half up, (sum + 128) >> 8, in exact integers.
* Columns: a neighbour left of column 0 or right of column W-1 takes the
  value of that edge column (clamp); only rows are skipped, as the paper says.
* Thres: strict |G_t - G_{t-1}| > t with t = 20, written as 255 (motion) or 0.
* Med: the median of the pixel and its 4 nearest neighbours (a plus shape);
  the outermost rows and columns are copied unchanged.
* Frame 0 is compared with the initial token (a zero frame unless given).

Everything is integer arithmetic, so the CUDA path must match bit for bit.
"""
from __future__ import annotations

import numpy as np

GAUSS_ROW = (1, 4, 6, 4, 1)
THRESHOLD = 20
MOTION = 255


def gauss5(frame: np.ndarray) -> np.ndarray:
    """5x5 binomial filter of rows 2 .. H-3 (columns clamped at the edges);
    rows 0, 1, H-2, H-1 are copied unfiltered."""
    f = np.asarray(frame, np.uint8)
    H, W = f.shape
    out = f.copy()
    if H <= 4:
        return out
    p = f.astype(np.int64)
    cols = np.clip(np.arange(-2, W + 2), 0, W - 1)       # clamped column index of x - 2 .. x + 2
    pc = p[:, cols]                                      # (H, W + 4)
    acc = np.zeros((H - 4, W), np.int64)
    for dy in range(5):
        for dx in range(5):
            acc += GAUSS_ROW[dy] * GAUSS_ROW[dx] * pc[dy:dy + H - 4, dx:dx + W]
    out[2:H - 2] = ((acc + 128) >> 8).astype(np.uint8)
    return out


def thres(cur: np.ndarray, prev: np.ndarray, t: int = THRESHOLD) -> np.ndarray:
    """255 where |cur - prev| > t, else 0."""
    d = np.abs(np.asarray(cur, np.int64) - np.asarray(prev, np.int64))
    return np.where(d > t, MOTION, 0).astype(np.uint8)


def med5(m: np.ndarray) -> np.ndarray:
    """Median of the plus-shaped 5-pixel neighbourhood; border pixels copied."""
    f = np.asarray(m, np.uint8)
    H, W = f.shape
    out = f.copy()
    if H <= 2 or W <= 2:
        return out
    five = np.stack([f[1:-1, 1:-1], f[:-2, 1:-1], f[2:, 1:-1], f[1:-1, :-2], f[1:-1, 2:]])
    out[1:-1, 1:-1] = np.sort(five, axis=0)[2]
    return out


def pipeline(frames: np.ndarray, t: int = THRESHOLD, initial: np.ndarray | None = None) -> np.ndarray:
    """Motion maps of a frame sequence: Med(Thres(Gauss(f_t), Gauss(f_{t-1}))), where the
    previous filtered frame of frame 0 is the initial token (zeros unless given)."""
    frames = np.asarray(frames, np.uint8)
    T, H, W = frames.shape
    prev = np.zeros((H, W), np.uint8) if initial is None else np.asarray(initial, np.uint8)
    out = np.empty_like(frames)
    for i in range(T):
        g = gauss5(frames[i])
        out[i] = med5(thres(g, prev, t))
        prev = g
    return out
