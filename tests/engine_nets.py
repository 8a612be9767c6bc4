"""Builders of the benchmark networks through the engine's C ABI (test helper).

They mirror ``oracle/nets.py`` port for port, so the same pushes and runs can
be replayed on both sides."""
import numpy as np

CPLX = 8


def dpd_fused(Net, h, orders, block_len, delay, capacity, out_capacity=None):
    net = Net()
    ids = {}
    ids["ctrl"] = net.add_source()
    ids["data"] = net.add_source()
    ids["dpd"] = net.add_dpd(h, orders, block_len)
    ids["sink"] = net.add_sink()
    blk = block_len * CPLX
    ids["ch_ctrl"] = net.connect(ids["ctrl"], 0, ids["dpd"], 0, 4, 1, capacity)
    ids["ch_data"] = net.connect(ids["data"], 0, ids["dpd"], 1, blk, 1, capacity, delay)
    ids["ch_out"] = net.connect(ids["dpd"], 0, ids["sink"], 0, blk, 1,
                                capacity if out_capacity is None else out_capacity)
    net.finalize()
    return net, ids


def motion_fused(Net, height, width, capacity, rec_capacity=None, t=25, prev_init=None,
                 separate_prev_source=False):
    n_tiles = (-(-height // 16)) * (-(-width // 16))
    net = Net()
    ids = {}
    ids["src"] = net.add_source()
    if separate_prev_source:
        ids["src_prev"] = net.add_source()
    ids["md"] = net.add_md(width, height, t)
    ids["rec"] = net.add_sink()
    ids["cnt"] = net.add_sink()
    fb = height * width
    ids["ch_cur"] = net.connect(ids["src"], 0, ids["md"], 0, fb, 1, capacity)
    psrc, pport = (ids["src_prev"], 0) if separate_prev_source else (ids["src"], 1)
    ids["ch_prev"] = net.connect(psrc, pport, ids["md"], 1, fb, 1, capacity, 1,
                                 None if prev_init is None else np.ascontiguousarray(prev_init))
    rc = capacity * n_tiles if rec_capacity is None else rec_capacity
    ids["ch_rec"] = net.connect(ids["md"], 0, ids["rec"], 0, 8, n_tiles, rc)
    ids["ch_cnt"] = net.connect(ids["md"], 1, ids["cnt"], 0, 4, 1, capacity)
    net.finalize()
    return net, ids


def dpd_expanded(Net, h, orders, block_len, delay, capacity, branch_capacity=None):
    """The Sec. 4.2 network on the engine: control source feeds Poly and Adder;
    Poly -> FIR_k -> Adder; same actor and channel order as the oracle's builder."""
    from paper_1611_03226_b300 import _lib as L
    K = len(orders)
    bc = capacity if branch_capacity is None else branch_capacity
    blk = block_len * CPLX
    net = Net()
    ids = {}
    ids["ctrl"] = net.add_source()
    ids["data"] = net.add_source()
    ids["poly"] = net.add_dpd(h, orders, block_len, kind=L.DF_DPD_POLY)
    ids["fir"] = [net.add_dpd(h, orders, block_len, kind=L.DF_DPD_FIR, branch=k) for k in range(K)]
    ids["add"] = net.add_dpd(h, orders, block_len, kind=L.DF_DPD_ADD)
    ids["sink"] = net.add_sink()
    net.connect(ids["ctrl"], 0, ids["poly"], 0, 4, 1, capacity)
    net.connect(ids["ctrl"], 1, ids["add"], 0, 4, 1, capacity)
    ids["ch_data"] = net.connect(ids["data"], 0, ids["poly"], 1, blk, 1, capacity, delay)
    for k in range(K):
        net.connect(ids["poly"], k, ids["fir"][k], 0, blk, 1, bc)
        net.connect(ids["fir"][k], 0, ids["add"], k + 1, blk, 1, bc)
    ids["ch_out"] = net.connect(ids["add"], 0, ids["sink"], 0, blk, 1, capacity)
    net.finalize()
    return net, ids


def dpd_batch(Net, chans, capacity, stream=None):
    """Independent predistorter channels in one network.  chans: list of
    (h, orders, block_len).  Returns (net, per-channel dict of ids)."""
    net = Net(stream=stream)
    ids = []
    for (h, orders, L) in chans:
        d = {}
        d["ctrl"] = net.add_source()
        d["data"] = net.add_source()
        d["dpd"] = net.add_dpd(h, orders, L)
        d["sink"] = net.add_sink()
        blk = L * CPLX
        net.connect(d["ctrl"], 0, d["dpd"], 0, 4, 1, capacity)
        net.connect(d["data"], 0, d["dpd"], 1, blk, 1, capacity)
        net.connect(d["dpd"], 0, d["sink"], 0, blk, 1, capacity)
        ids.append(d)
    net.finalize()
    return net, ids


def motion_paper(Net, height, width, capacity, rate=1, t=20, initial=None, stream=None):
    """The paper's motion pipeline through the engine: Src -> Gauss -> {Thres in 0, Thres in 1
    with one initial frame} -> Med -> Sink, `rate` frames per firing on every channel."""
    net = Net(stream=stream) if stream is not None else Net()
    fb = height * width
    ids = {"src": net.add_source(), "gauss": net.add_gauss5(width, height),
           "thres": net.add_thres(width, height, t), "med": net.add_med5(width, height),
           "sink": net.add_sink()}
    init = None if initial is None else np.ascontiguousarray(initial, np.uint8)
    ids["ch_in"] = net.connect(ids["src"], 0, ids["gauss"], 0, fb, rate, capacity)
    ids["ch_cur"] = net.connect(ids["gauss"], 0, ids["thres"], 0, fb, rate, capacity)
    ids["ch_prev"] = net.connect(ids["gauss"], 1, ids["thres"], 1, fb, rate, capacity, 1, init)
    ids["ch_map"] = net.connect(ids["thres"], 0, ids["med"], 0, fb, rate, capacity)
    ids["ch_out"] = net.connect(ids["med"], 0, ids["sink"], 0, fb, rate, capacity)
    net.finalize()
    return net, ids
