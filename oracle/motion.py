"""Motion-detection arithmetic on exact integers (oracle; test infrastructure).

Pipeline (the benchmark variant of the Sec. 4.1 application): absolute
difference of consecutive frames (the previous frame arrives through a channel
holding one initial token), threshold, 3x3 binary erosion then 3x3 binary
dilation (an opening), then one record per 16x16 tile that contains motion.

Readings adopted where the text is silent:
* threshold is strict: pixel is 1 iff |cur - prev| > t (t = 25);
* morphology counts in-frame neighbours only: erosion treats pixels outside
  the frame as 1, dilation treats them as 0;
* tiles are 16x16 in raster order (tile row, then tile column); a partial
  last row/column of tiles covers only in-frame pixels; a record
  (16*tx, 16*ty, count) is emitted iff count > 0.
"""
from __future__ import annotations

import numpy as np

RECORD_DTYPE = np.dtype([("x", "<u2"), ("y", "<u2"), ("count", "<u4")])


def absdiff(cur: np.ndarray, prev: np.ndarray) -> np.ndarray:
    return np.abs(cur.astype(np.int16) - prev.astype(np.int16)).astype(np.uint8)


def threshold(d: np.ndarray, t: int = 25) -> np.ndarray:
    return (d > t).astype(np.uint8)


def _neighbourhood(b: np.ndarray, border: int, combine):
    H, W = b.shape
    p = np.full((H + 2, W + 2), border, np.uint8)
    p[1:-1, 1:-1] = b
    out = p[1:H + 1, 1:W + 1].copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out = combine(out, p[1 + dy:H + 1 + dy, 1 + dx:W + 1 + dx])
    return out


def erode3x3(b: np.ndarray) -> np.ndarray:
    """3x3 erosion; out-of-frame neighbours count as 1."""
    return _neighbourhood(b, 1, np.minimum)


def dilate3x3(b: np.ndarray) -> np.ndarray:
    """3x3 dilation; out-of-frame neighbours count as 0."""
    return _neighbourhood(b, 0, np.maximum)


def tile_counts(o: np.ndarray, tile: int = 16) -> np.ndarray:
    """Number of set pixels in each tile x tile tile (partial edge tiles allowed)."""
    H, W = o.shape
    th, tw = -(-H // tile), -(-W // tile)
    p = np.zeros((th * tile, tw * tile), np.uint32)
    p[:H, :W] = o
    return p.reshape(th, tile, tw, tile).sum(axis=(1, 3), dtype=np.uint32)


def tile_records(counts: np.ndarray, tile: int = 16) -> np.ndarray:
    """Records of the tiles with motion, raster order."""
    ty, tx = np.nonzero(counts)          # row-major = raster order
    rec = np.empty(len(ty), RECORD_DTYPE)
    rec["x"] = tx * tile
    rec["y"] = ty * tile
    rec["count"] = counts[ty, tx]
    return rec


def detect(cur: np.ndarray, prev: np.ndarray, t: int = 25, tile: int = 16) -> np.ndarray:
    """The five stages composed: records for one frame."""
    return tile_records(tile_counts(dilate3x3(erode3x3(threshold(absdiff(cur, prev), t))), tile), tile)
