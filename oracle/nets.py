"""Builders for the benchmark networks on the oracle interpreter (test infrastructure)."""
from __future__ import annotations

import numpy as np

from . import actors as A
from .network import Network, Sink, Source

CPLX = 8     # bytes per complex64 sample


def dpd_fused(h, orders, block_len, delay, capacity, record_history=False):
    """ctrl source -> DPD.in0, data source -(delay zero blocks)-> DPD.in1, DPD -> sink.

    Returns (net, ids) with ids = dict(ctrl, data, dpd, sink, ch_ctrl, ch_data, ch_out).
    """
    net = Network(record_history)
    ids = {}
    ids["ctrl"] = net.add_actor(Source())
    ids["data"] = net.add_actor(Source())
    ids["dpd"] = net.add_actor(A.Dpd(h, orders, block_len))
    ids["sink"] = net.add_actor(Sink())
    zero = np.zeros(block_len, np.complex128)
    ids["ch_ctrl"] = net.connect(ids["ctrl"], 0, ids["dpd"], 0, 1, capacity, token_bytes=4)
    ids["ch_data"] = net.connect(ids["data"], 0, ids["dpd"], 1, 1, capacity,
                                 [zero.copy() for _ in range(delay)], token_bytes=block_len * CPLX)
    ids["ch_out"] = net.connect(ids["dpd"], 0, ids["sink"], 0, 1, capacity,
                                token_bytes=block_len * CPLX)
    net.finalize()
    return net, ids


def dpd_expanded(h, orders, block_len, delay, capacity, branch_capacity=None,
                 record_history=False):
    """The Sec. 4.2 network: ctrl source feeds Poly and Adder; Poly -> FIR_k -> Adder."""
    K = len(orders)
    bc = capacity if branch_capacity is None else branch_capacity
    net = Network(record_history)
    ids = {}
    ids["ctrl"] = net.add_actor(Source())
    ids["data"] = net.add_actor(Source())
    ids["poly"] = net.add_actor(A.DpdPoly(orders))
    ids["fir"] = [net.add_actor(A.DpdFir(h[k])) for k in range(K)]
    ids["add"] = net.add_actor(A.DpdAdd(K, block_len))
    ids["sink"] = net.add_actor(Sink())
    zero = np.zeros(block_len, np.complex128)
    net.connect(ids["ctrl"], 0, ids["poly"], 0, 1, capacity, token_bytes=4)
    net.connect(ids["ctrl"], 1, ids["add"], 0, 1, capacity, token_bytes=4)
    ids["ch_data"] = net.connect(ids["data"], 0, ids["poly"], 1, 1, capacity,
                                 [zero.copy() for _ in range(delay)], token_bytes=block_len * CPLX)
    for k in range(K):
        net.connect(ids["poly"], k, ids["fir"][k], 0, 1, bc, token_bytes=block_len * CPLX)
        net.connect(ids["fir"][k], 0, ids["add"], k + 1, 1, bc, token_bytes=block_len * CPLX)
    ids["ch_out"] = net.connect(ids["add"], 0, ids["sink"], 0, 1, capacity,
                                token_bytes=block_len * CPLX)
    net.finalize()
    return net, ids


def as_tokens_ctrl(masks):
    return [np.uint32(m) for m in masks]


def as_tokens_blocks(blocks):
    return [np.asarray(b) for b in blocks]


def motion_fused(height, width, capacity, rec_capacity=None, t=25, tile=16,
                 prev_init=None, record_history=False):
    """frames source -> (cur, prev with one initial frame) -> Md -> records / counts sinks."""
    n_tiles = (-(-height // tile)) * (-(-width // tile))
    net = Network(record_history)
    ids = {}
    ids["src"] = net.add_actor(Source())
    ids["md"] = net.add_actor(A.Md(t, tile))
    ids["rec"] = net.add_actor(Sink())
    ids["cnt"] = net.add_actor(Sink())
    fb = height * width
    init = np.zeros((height, width), np.uint8) if prev_init is None else prev_init
    ids["ch_cur"] = net.connect(ids["src"], 0, ids["md"], 0, 1, capacity, token_bytes=fb)
    ids["ch_prev"] = net.connect(ids["src"], 1, ids["md"], 1, 1, capacity, [init.copy()],
                                 token_bytes=fb)
    rc = capacity * n_tiles if rec_capacity is None else rec_capacity
    ids["ch_rec"] = net.connect(ids["md"], 0, ids["rec"], 0, n_tiles, rc, token_bytes=8)
    ids["ch_cnt"] = net.connect(ids["md"], 1, ids["cnt"], 0, 1, capacity, token_bytes=4)
    net.finalize()
    return net, ids


def motion_literal(height, width, capacity, rec_capacity=None, t=25, tile=16,
                   prev_init=None, record_history=False):
    """Diff -> Thresh -> Erode -> Dilate -> Tiles as five actors with frame channels."""
    n_tiles = (-(-height // tile)) * (-(-width // tile))
    net = Network(record_history)
    ids = {}
    ids["src"] = net.add_actor(Source())
    ids["diff"] = net.add_actor(A.MdDiff())
    ids["thr"] = net.add_actor(A.MdThresh(t))
    ids["ero"] = net.add_actor(A.MdErode())
    ids["dil"] = net.add_actor(A.MdDilate())
    ids["tiles"] = net.add_actor(A.MdTiles(tile))
    ids["rec"] = net.add_actor(Sink())
    ids["cnt"] = net.add_actor(Sink())
    fb = height * width
    init = np.zeros((height, width), np.uint8) if prev_init is None else prev_init
    ids["ch_cur"] = net.connect(ids["src"], 0, ids["diff"], 0, 1, capacity, token_bytes=fb)
    ids["ch_prev"] = net.connect(ids["src"], 1, ids["diff"], 1, 1, capacity, [init.copy()],
                                 token_bytes=fb)
    net.connect(ids["diff"], 0, ids["thr"], 0, 1, capacity, token_bytes=fb)
    net.connect(ids["thr"], 0, ids["ero"], 0, 1, capacity, token_bytes=fb)
    net.connect(ids["ero"], 0, ids["dil"], 0, 1, capacity, token_bytes=fb)
    net.connect(ids["dil"], 0, ids["tiles"], 0, 1, capacity, token_bytes=fb)
    rc = capacity * n_tiles if rec_capacity is None else rec_capacity
    ids["ch_rec"] = net.connect(ids["tiles"], 0, ids["rec"], 0, n_tiles, rc, token_bytes=8)
    ids["ch_cnt"] = net.connect(ids["tiles"], 1, ids["cnt"], 0, 1, capacity, token_bytes=4)
    net.finalize()
    return net, ids


def records_of(tokens):
    """Concatenate popped record tokens into one structured array."""
    from .motion import RECORD_DTYPE
    if not tokens:
        return np.empty(0, RECORD_DTYPE)
    return np.concatenate([np.asarray(t, RECORD_DTYPE).reshape(-1) for t in tokens])


def motion_paper(height, width, capacity, rate=1, t=20, initial=None, record_history=False):
    """The paper's motion pipeline (Sec. 4.1): Src -> Gauss -> {Thres in 0, Thres in 1 with one
    initial frame} -> Med -> Sink, every channel carrying `rate` frames per firing."""
    net = Network(record_history)
    ids = {}
    ids["src"] = net.add_actor(Source())
    ids["gauss"] = net.add_actor(A.Gauss5())
    ids["thres"] = net.add_actor(A.Thres(t))
    ids["med"] = net.add_actor(A.Med5())
    ids["sink"] = net.add_actor(Sink())
    fb = height * width
    init = np.zeros((height, width), np.uint8) if initial is None else np.asarray(initial, np.uint8)
    ids["ch_in"] = net.connect(ids["src"], 0, ids["gauss"], 0, rate, capacity, token_bytes=fb)
    ids["ch_cur"] = net.connect(ids["gauss"], 0, ids["thres"], 0, rate, capacity, token_bytes=fb)
    ids["ch_prev"] = net.connect(ids["gauss"], 1, ids["thres"], 1, rate, capacity, [init.copy()],
                                 token_bytes=fb)
    ids["ch_map"] = net.connect(ids["thres"], 0, ids["med"], 0, rate, capacity, token_bytes=fb)
    ids["ch_out"] = net.connect(ids["med"], 0, ids["sink"], 0, rate, capacity, token_bytes=fb)
    net.finalize()
    return net, ids
