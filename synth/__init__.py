"""Seeded synthetic inputs shaped like the paper's two workloads.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no predistortion, no motion detection, no dataflow
semantics).  Both the CPU oracle and the CUDA path take their inputs from here,
so the two sides always see identical arrays.

Workloads (all complex data is complex64 = interleaved float32 I/Q):

* ``dpd_tiny``   64 blocks x 4096 samples, up to 4 branches of order 1,3,5,7,
                 10 taps, per-block control picks a prefix of 1-4 branches.
* ``dpd_large``  512 blocks x 2^20 samples, up to 8 branches of odd order 1-15,
                 16 taps, per-block control mask uniform in 1..255.
* ``dpd_batch``  256 independent channels, log-uniform block length 1 Ki-256 Ki,
                 per-channel static branch mask, 8-16 taps.
* ``dpd_fit``    2^18 samples for the indirect-learning fit.
* ``motion``     1920x1080 uint8 frames: textured background, 1-8 moving
                 rectangles, clipped Gaussian noise.

Every generator is a pure function of ``seed`` (numpy PCG64 via
``default_rng``); block-wise generators seed each block separately so that any
subset can be regenerated without producing the whole stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1611032260

#: record layout of one emitted motion tile: 8 bytes, little endian
RECORD_DTYPE = np.dtype([("x", "<u2"), ("y", "<u2"), ("count", "<u4")])


def _cplx(rng: np.random.Generator, shape, std: float) -> np.ndarray:
    """complex64 with independent N(0, std) real and imaginary parts."""
    a = rng.standard_normal(tuple(shape) + (2,), dtype=np.float32)
    a *= np.float32(std)
    return a.view(np.complex64).reshape(shape)


# --------------------------------------------------------------------------
# predistortion workloads
# --------------------------------------------------------------------------
@dataclass
class DpdWorkload:
    """One dynamic predistortion stream.

    ``masks[i]`` is the control token of firing i (bit k = branch k active).
    ``h[k, m]`` is tap m of branch k; branch k applies polynomial order
    ``orders[k]``.  Blocks are produced lazily by :meth:`block`.
    """
    name: str
    seed: int
    n_blocks: int
    block_len: int
    orders: tuple
    n_taps: int
    h: np.ndarray            # (K, M) complex64
    masks: np.ndarray        # (n_blocks,) uint32
    delay: int               # initial (delay) data blocks
    capacity: int            # FIFO capacity in blocks used by the workload
    x_std: float = 0.3

    @property
    def n_branches(self) -> int:
        return len(self.orders)

    def block(self, b: int) -> np.ndarray:
        """Input block b (complex64, ``block_len`` samples)."""
        rng = np.random.default_rng([self.seed, 1, b])
        return _cplx(rng, (self.block_len,), self.x_std)

    def blocks(self, start: int = 0, stop: int | None = None) -> np.ndarray:
        stop = self.n_blocks if stop is None else stop
        out = np.empty((stop - start, self.block_len), np.complex64)
        for i, b in enumerate(range(start, stop)):
            out[i] = self.block(b)
        return out


def _coeffs(rng, K, M, std=0.1):
    h = _cplx(rng, (K, M), std)
    h[0, 0] = 1.0 + 0.0j          # linear branch, first tap: unit gain
    return h


def dpd_tiny(seed: int = BASE_SEED + 0) -> DpdWorkload:
    """64 blocks x 4096, K<=4 (orders 1,3,5,7), M=10, prefix masks, d=1, capacity 8."""
    rng = np.random.default_rng([seed, 0])
    h = _coeffs(rng, 4, 10)
    c = rng.integers(1, 5, size=64)                 # 1..4 active branches
    masks = ((np.uint32(1) << c.astype(np.uint32)) - np.uint32(1)).astype(np.uint32)
    return DpdWorkload("dpd_tiny_64x4096", seed, 64, 4096, (1, 3, 5, 7), 10, h,
                       masks, delay=1, capacity=8)


def dpd_large(seed: int = BASE_SEED + 2, n_blocks: int = 512,
              block_len: int = 1 << 20) -> DpdWorkload:
    """512 blocks x 2^20, K<=8 (orders 1..15), M=16, masks U{1..255}, d=2."""
    rng = np.random.default_rng([seed, 0])
    h = _coeffs(rng, 8, 16)
    masks = rng.integers(1, 256, size=n_blocks).astype(np.uint32)
    return DpdWorkload(f"dpd_large_{n_blocks}x{block_len}", seed, n_blocks, block_len,
                       tuple(range(1, 16, 2)), 16, h, masks, delay=2,
                       capacity=n_blocks + 2)


def log_uniform_lengths(rng, n, lo=1024, hi=262144) -> np.ndarray:
    """L = floor(exp(U(ln lo, ln hi)))."""
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(np.int64)


@dataclass
class DpdBatchWorkload:
    """Independent predistortion channels with uneven sizes (batched launch)."""
    name: str
    seed: int
    lengths: np.ndarray      # (C,) block length per channel
    taps: np.ndarray         # (C,) M per channel
    masks: np.ndarray        # (C,) static branch mask per channel
    h: list                  # per channel (8, M_c) complex64
    orders: tuple = tuple(range(1, 16, 2))
    blocks_per_channel: int = 16

    @property
    def n_channels(self) -> int:
        return len(self.lengths)

    def block(self, c: int, b: int) -> np.ndarray:
        rng = np.random.default_rng([self.seed, 2, c, b])
        return _cplx(rng, (int(self.lengths[c]),), 0.3)


def dpd_batch(seed: int = BASE_SEED + 3, n_channels: int = 256,
              blocks_per_channel: int = 16) -> DpdBatchWorkload:
    rng = np.random.default_rng([seed, 0])
    lengths = log_uniform_lengths(rng, n_channels)
    taps = rng.integers(8, 17, size=n_channels)
    masks = rng.integers(1, 256, size=n_channels).astype(np.uint32)
    h = [_coeffs(rng, 8, int(m)) for m in taps]
    return DpdBatchWorkload(f"dpd_batch_{n_channels}ch", seed, lengths, taps, masks, h,
                            blocks_per_channel=blocks_per_channel)


@dataclass
class DpdFitWorkload:
    seed: int
    x: np.ndarray            # (N,) complex64
    orders: tuple = (1, 3, 5, 7)
    n_taps: int = 10
    steps: int = 200
    lr: float = 1e-3
    # Saleh AM/AM (alpha_a, beta_a), AM/PM (alpha_p, beta_p), 3-tap memory FIR
    saleh: tuple = (2.1587, 1.1517, 4.0033, 9.1040)
    memory: tuple = (1.0, 0.1, -0.05)


def dpd_fit(seed: int = BASE_SEED + 4, n: int = 1 << 18) -> DpdFitWorkload:
    rng = np.random.default_rng([seed, 0])
    return DpdFitWorkload(seed, _cplx(rng, (n,), 0.3))


# --------------------------------------------------------------------------
# motion-detection workload
# --------------------------------------------------------------------------
@dataclass
class MotionWorkload:
    """Grayscale video: ``frame(t)`` returns frame t as (H, W) uint8."""
    name: str
    seed: int
    n_frames: int
    height: int
    width: int
    background: np.ndarray = field(repr=False)
    rects: list = field(repr=False)      # [(x, y, w, h, vx, vy, gray)]
    noise: bool = True
    noise_std: float = 20.0 / 3.0

    def _positions(self, t: int):
        """Rectangle positions at frame t; bouncing at the frame edges."""
        out = []
        for (x0, y0, w, h, vx, vy, g) in self.rects:
            out.append((_bounce(x0, vx, t, self.width - w), _bounce(y0, vy, t, self.height - h), w, h, g))
        return out

    def frame(self, t: int) -> np.ndarray:
        f = self.background.copy()
        for (x, y, w, h, g) in self._positions(t):
            f[y:y + h, x:x + w] = g
        if self.noise:
            rng = np.random.default_rng([self.seed, 3, t])
            nz = rng.standard_normal(f.shape, dtype=np.float32)
            nz *= np.float32(self.noise_std)
            np.rint(nz, out=nz)
            np.clip(nz, -20, 20, out=nz)
            f = f.astype(np.int16) + nz.astype(np.int16)
        return np.clip(f, 0, 255).astype(np.uint8)

    def frames(self, start: int = 0, stop: int | None = None) -> np.ndarray:
        stop = self.n_frames if stop is None else stop
        out = np.empty((stop - start, self.height, self.width), np.uint8)
        for i, t in enumerate(range(start, stop)):
            out[i] = self.frame(t)
        return out


def _bounce(p0: int, v: int, t: int, span: int) -> int:
    """Position at time t of a point moving with speed v on [0, span], reflecting."""
    if span <= 0:
        return 0
    period = 2 * span
    q = (p0 + v * t) % period
    return int(q if q <= span else period - q)


def _texture(rng, H, W) -> np.ndarray:
    """Background in [40, 200]: three random sinusoids plus box-smoothed noise."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float32)
    acc = np.zeros((H, W), np.float32)
    for _ in range(3):
        fx, fy = rng.uniform(0.002, 0.03, size=2)
        ph = rng.uniform(0, 2 * np.pi)
        acc += np.sin(2 * np.pi * (fx * xx + fy * yy) + ph).astype(np.float32)
    nz = rng.standard_normal((H // 8 + 1, W // 8 + 1), dtype=np.float32)
    nz = np.kron(nz, np.ones((8, 8), np.float32))[:H, :W]     # blocky, then smoothed
    k = 9
    c = np.cumsum(np.cumsum(np.pad(nz, ((k, k), (k, k)), mode="edge"), 0), 1)
    sm = (c[2 * k:, 2 * k:] - c[:-2 * k, 2 * k:] - c[2 * k:, :-2 * k] + c[:-2 * k, :-2 * k])
    sm = sm[:H, :W] / np.float32((2 * k) ** 2)
    acc += 2.0 * sm
    lo, hi = float(acc.min()), float(acc.max())
    return (40.0 + 160.0 * (acc - lo) / max(hi - lo, 1e-6)).round().astype(np.uint8)


def motion(seed: int = BASE_SEED + 1, n_frames: int = 300, height: int = 1080,
           width: int = 1920, noise: bool = True) -> MotionWorkload:
    rng = np.random.default_rng([seed, 0])
    bg = _texture(rng, height, width)
    rects = []
    for _ in range(int(rng.integers(1, 9))):
        w, h = (int(v) for v in rng.integers(32, 401, size=2))
        w, h = min(w, width), min(h, height)
        x0 = int(rng.integers(0, width - w + 1))
        y0 = int(rng.integers(0, height - h + 1))
        vx, vy = (int(v) for v in rng.integers(-8, 9, size=2))
        local = float(bg[y0:y0 + h, x0:x0 + w].mean())
        step = float(rng.uniform(40, 90))
        g = local + step if rng.random() < 0.5 else local - step
        if g > 255 or g < 0:                 # keep at least 40 levels of contrast
            g = local - step if g > 255 else local + step
        rects.append((x0, y0, w, h, vx, vy, int(np.clip(round(g), 0, 255))))
    return MotionWorkload(f"motion_{n_frames}x{width}x{height}", seed, n_frames, height,
                          width, bg, rects, noise)


def flat_with_rect(height: int, width: int, n_frames: int, rect_w: int, rect_h: int,
                   x0: int, y0: int, dx: int, bg: int = 100, fg: int = 180) -> np.ndarray:
    """Noise-free frames: flat background, one rectangle moving by (dx, 0) per frame."""
    out = np.full((n_frames, height, width), bg, np.uint8)
    for t in range(n_frames):
        x = x0 + dx * t
        out[t, y0:y0 + rect_h, max(x, 0):max(x + rect_w, 0)] = fg
    return out


def uniform_frames(n_frames: int, height: int, width: int, seed: int = BASE_SEED + 5) -> np.ndarray:
    """Frames of independent uniform bytes: pixel differences cover 0..255, so
    every threshold has pixels just below, at and just above it."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(n_frames, height, width), dtype=np.uint8)


def blocky_frames(n_frames: int, height: int, width: int, block: int = 4,
                  seed: int = BASE_SEED + 6) -> np.ndarray:
    """Frames of uniform random bytes constant over block x block squares: with
    high thresholds the motion mask keeps areas that survive the 3x3 erosion."""
    rng = np.random.default_rng(seed)
    hb, wb = -(-height // block), -(-width // block)
    small = rng.integers(0, 256, size=(n_frames, hb, wb), dtype=np.uint8)
    return np.repeat(np.repeat(small, block, axis=1), block, axis=2)[:, :height, :width].copy()
