"""Parity of the fused predistorter actor (CUDA, FP32) with the float64 oracle.

Both sides receive the same pushes and runs; because a step of the engine and
a sweep of the oracle fire the same firings, channel counters agree after
every step, and each output block matches within 1e-5 relative L2."""
import numpy as np
import pytest

import engine_nets as EN
import synth
from oracle import dpd as D
from oracle import nets as ON

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def Net():
    from paper_1611_03226_b300 import Net
    return Net


def stream_both(Net, h, orders, L, d, cap, masks, blocks, chunk, rng=None, tile=None, flags=0):
    onet, oi = ON.dpd_fused(h, orders, L, d, cap)
    enet, ei = EN.dpd_fused(Net, h, orders, L, d, cap)
    if tile:
        enet.set_tile(ei["dpd"], *tile)
    yo, ye = [], []
    n, i, idle = len(masks), 0, 0
    while True:
        free = min(onet.channels[oi["ch_ctrl"]].free, onet.channels[oi["ch_data"]].free)
        k = min(chunk, n - i, free)
        if k > 0:
            onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks[i:i + k]))
            onet.push(oi["data"], ON.as_tokens_blocks(blocks[i:i + k]))
            enet.push(ei["ctrl"], np.ascontiguousarray(masks[i:i + k], np.uint32))
            enet.push(ei["data"], np.ascontiguousarray(blocks[i:i + k], np.complex64))
            i += k
        steps = 1 if rng is None else int(rng.integers(1, 3))
        fo = onet.run(steps)
        fe = enet.run(steps, flags)
        assert fo == fe
        for key in ("ch_ctrl", "ch_data", "ch_out"):
            assert onet.counters(oi[key]) == enet.counters(ei[key])
        m = int(rng.integers(0, 3)) if rng is not None else None
        yo += onet.pop(oi["sink"], m)
        ye.append(enet.pop(ei["sink"], m, dtype=np.complex64))
        if i >= n and fo == 0:
            idle += 1
            if idle > 2 and not onet.channels[oi["ch_out"]].occupancy:
                break
    enet.close()
    return np.array(yo).reshape(-1, L), np.concatenate(ye).reshape(-1, L)


def check_blocks(yo, ye, tol=TOL):
    assert yo.shape == ye.shape
    errs = [D.rel_l2(ye[b], yo[b]) for b in range(len(yo))]
    assert max(errs) <= tol, (max(errs), int(np.argmax(errs)))
    return max(errs)


def test_identity_predistorter_exact(Net):
    rng = np.random.default_rng(1)
    L, n = 600, 11
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = np.zeros((4, 10), np.complex64)
    h[0, 0] = 1
    masks = (rng.integers(0, 16, n) | 1).astype(np.uint32)
    yo, ye = stream_both(Net, h, (1, 3, 5, 7), L, 2, 4, masks, x, 2)
    want = np.concatenate([np.zeros((2, L), np.complex64), x[:-2]])
    np.testing.assert_array_equal(ye, want)
    np.testing.assert_array_equal(yo, want)


def test_tiny_workload_full_size(Net):
    """64 blocks x 4096, K<=4, M=10, prefix masks, capacity 8, one delay block."""
    w = synth.dpd_tiny()
    yo, ye = stream_both(Net, w.h, w.orders, w.block_len, w.delay, w.capacity, w.masks,
                         w.blocks(), 3)
    assert len(ye) == 64
    check_blocks(yo, ye)


@pytest.mark.parametrize("L,M,d,K,cap,tile", [
    (64, 10, 1, 4, 5, None),          # short blocks, one tile
    (3, 10, 2, 8, 6, None),           # block shorter than the FIR history
    (1, 4, 0, 3, 4, None),            # single-sample blocks
    (5000, 16, 2, 8, 7, (1024, 128)),  # ragged last tile, several tiles per block
    (2047, 32, 1, 5, 4, (2048, 256)),  # two 16-tap chunks
    (777, 13, 3, 16, 9, (1024, 64)),  # 16 branches, odd tap count
    (4096, 9, 1, 6, 5, (2048, 128)),  # R = 16 variant
    (3000, 11, 2, 4, 6, (256, 32)),   # one-warp CTAs, the autotuner's smallest tile
])
def test_random_masks_parity(Net, L, M, d, K, cap, tile):
    rng = np.random.default_rng(L + 7 * M + K)
    n = 14
    orders = tuple(range(1, 2 * K, 2))
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    masks = rng.integers(0, 1 << K, n).astype(np.uint32)
    masks[3] = 0                        # an empty mask gives a zero block
    yo, ye = stream_both(Net, h, orders, L, d, cap, masks, x, 3, rng=rng, tile=tile)
    assert len(ye) == n
    check_blocks(yo, ye)


def test_mask_bits_beyond_K_ignored(Net):
    rng = np.random.default_rng(5)
    L, n = 100, 6
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, .1, (2, 5)) + 1j * rng.normal(0, .1, (2, 5))).astype(np.complex64)
    masks = np.array([0xFFFFFFFF, 4, 1, 2, 0xF0, 3], np.uint32)
    yo, ye = stream_both(Net, h, (1, 3), L, 0, 8, masks, x, 6)
    check_blocks(yo, ye)


def test_stateless_forward_backward(Net):
    import torch
    from paper_1611_03226_b300 import dpd as G
    rng = np.random.default_rng(9)
    for n, K, M in ((20000, 4, 10), (3001, 3, 32), (1, 2, 5)):
        orders = tuple(range(1, 2 * K, 2))
        x = (rng.normal(0, .3, n) + 1j * rng.normal(0, .3, n)).astype(np.complex64)
        h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
        g = (rng.normal(size=n) + 1j * rng.normal(size=n)).astype(np.complex64)
        xt, ht, gt = (torch.from_numpy(a).cuda() for a in (x, h, g))
        y = G.dpd_forward(xt, ht, orders).cpu().numpy()
        assert D.rel_l2(y, D.dpd_stream(x, h, orders)) <= TOL
        gx, gh = G.dpd_backward(xt, ht, orders, gt)
        rx, rh = D.dpd_stream_backward(x, h, orders, g)
        assert D.rel_l2(gx.cpu().numpy(), rx) <= 1e-3
        assert D.rel_l2(gh.cpu().numpy(), rh) <= 1e-3
        gx2, gh2 = G.dpd_backward(xt, ht, orders, gt)       # deterministic reduction
        assert torch.equal(gh, gh2) and torch.equal(gx, gx2)


@pytest.mark.parametrize("L,M,K,d,bc", [(512, 10, 4, 1, 2), (3, 6, 3, 2, 1), (2000, 16, 8, 1, 3)])
@pytest.mark.parametrize("persistent", [False, True])
def test_expanded_network_step_by_step(Net, L, M, K, d, bc, persistent):
    """The paper's Poly -> FIR_k -> Adder network with dynamic per-firing branch
    rates: every channel's counters equal the oracle's after every step, and
    the output stream matches within 1e-5 per block."""
    rng = np.random.default_rng(L + K)
    n = 10
    orders = tuple(range(1, 2 * K, 2))
    x = (rng.normal(0, .3, (n, L)) + 1j * rng.normal(0, .3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    masks = rng.integers(0, 1 << K, n).astype(np.uint32)
    cap = 4
    onet, oi = ON.dpd_expanded(h, orders, L, d, cap, branch_capacity=bc)
    enet, ei = EN.dpd_expanded(Net, h, orders, L, d, cap, branch_capacity=bc)
    i = 0
    yo, ye = [], []
    for step in range(200):
        free = min(onet.channels[0].free, onet.channels[1].free, onet.channels[oi["ch_data"]].free)
        k = min(2, n - i, free)
        if k > 0:
            onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks[i:i + k]))
            onet.push(oi["data"], ON.as_tokens_blocks(x[i:i + k]))
            enet.push(ei["ctrl"], np.ascontiguousarray(masks[i:i + k]))
            enet.push(ei["data"], np.ascontiguousarray(x[i:i + k]))
            i += k
        from paper_1611_03226_b300 import _lib as Lb
        fo, fe = onet.run(1), enet.run(1, Lb.DF_RUN_PERSISTENT if persistent else 0)
        assert fo == fe, step
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
    check_blocks(yo, ye)


def test_batched_channels_match_oracle_and_per_channel_launches(Net):
    """Uneven channels in one network: the batched launch, one launch per
    channel, a CUDA-graph replay and the autotuned configuration all give each
    channel's oracle output."""
    from paper_1611_03226_b300 import _lib as L
    rng = np.random.default_rng(77)
    C, nb = 12, 3
    orders = tuple(range(1, 16, 2))
    chans, data, masks = [], [], []
    for c in range(C):
        Lc = int(rng.integers(700, 5000))
        M = int(rng.integers(8, 17))
        h = (rng.normal(0, .1, (8, M)) + 1j * rng.normal(0, .1, (8, M))).astype(np.complex64)
        chans.append((h, orders, Lc))
        data.append((rng.normal(0, .3, (nb, Lc)) + 1j * rng.normal(0, .3, (nb, Lc))).astype(np.complex64))
        masks.append(np.full(nb, int(rng.integers(1, 256)), np.uint32))
    want = []
    for c in range(C):
        onet, oi = ON.dpd_fused(chans[c][0], orders, chans[c][2], 0, nb)
        onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks[c]))
        onet.push(oi["data"], ON.as_tokens_blocks(data[c]))
        onet.run(-1)
        want.append(np.array(onet.pop(oi["sink"])))

    def run_once(flags, tune=False):
        net, ids = EN.dpd_batch(Net, chans, nb)
        for c in range(C):
            net.push(ids[c]["ctrl"], masks[c])
            net.push(ids[c]["data"], data[c])
        if tune:
            assert net.autotune() == C * nb
            t = net.get_tile(ids[0]["dpd"])
            assert t[0] > 0 and t[1] > 0
        else:
            assert net.run(1, flags) == C * nb
        outs = [net.pop(ids[c]["sink"], dtype=np.complex64).reshape(nb, -1) for c in range(C)]
        net.close()
        return outs

    variants = {"batched": run_once(0), "per_channel": run_once(L.DF_RUN_NO_BATCH),
                "graph": run_once(L.DF_RUN_GRAPH), "autotuned": run_once(0, tune=True),
                "persistent": run_once(L.DF_RUN_PERSISTENT),
                "persistent_graph": run_once(L.DF_RUN_PERSISTENT | L.DF_RUN_GRAPH)}
    for name, outs in variants.items():
        for c in range(C):
            check_blocks(want[c], outs[c])
    for c in range(C):
        np.testing.assert_array_equal(variants["batched"][c], variants["per_channel"][c])
        np.testing.assert_array_equal(variants["batched"][c], variants["graph"][c])


@pytest.mark.parametrize("graph", [False, True])
def test_persistent_mode_streams_tiny_workload(Net, graph):
    """The 64 x 4096 workload through capacity-8 FIFOs, every step one
    persistent-kernel launch (replayed from a CUDA graph, or launched)."""
    from paper_1611_03226_b300 import _lib as L
    w = synth.dpd_tiny()
    flags = L.DF_RUN_PERSISTENT | (L.DF_RUN_GRAPH if graph else 0)
    yo, ye = stream_both(Net, w.h, w.orders, w.block_len, w.delay, w.capacity, w.masks,
                         w.blocks(), 3, flags=flags)
    assert len(ye) == 64
    check_blocks(yo, ye)


def test_persistent_run_to_quiescence_on_device(Net):
    """run(-1) in persistent mode: the quiescence test happens on the device."""
    from paper_1611_03226_b300 import _lib as L
    rng = np.random.default_rng(8)
    L_, n, K, M = 300, 9, 4, 10
    x = (rng.normal(0, .3, (n, L_)) + 1j * rng.normal(0, .3, (n, L_))).astype(np.complex64)
    h = (rng.normal(0, .1, (K, M)) + 1j * rng.normal(0, .1, (K, M))).astype(np.complex64)
    masks = rng.integers(0, 16, n).astype(np.uint32)
    orders = (1, 3, 5, 7)
    onet, oi = ON.dpd_expanded(h, orders, L_, 1, n + 1, branch_capacity=2)
    enet, ei = EN.dpd_expanded(Net, h, orders, L_, 1, n + 1, branch_capacity=2)
    onet.push(oi["ctrl"], ON.as_tokens_ctrl(masks))
    onet.push(oi["data"], ON.as_tokens_blocks(x))
    enet.push(ei["ctrl"], masks)
    enet.push(ei["data"], x)
    assert onet.run(-1) == enet.run(-1, L.DF_RUN_PERSISTENT)
    for c in range(len(onet.channels)):
        assert onet.counters(c) == enet.counters(c)
    yo = np.array(onet.pop(oi["sink"])).reshape(-1, L_)
    ye = enet.pop(ei["sink"], dtype=np.complex64).reshape(-1, L_)
    enet.close()
    check_blocks(yo, ye)


def test_bounded_wait_times_out_and_network_stays_usable(Net):
    """A grid barrier that waits for a CTA that never arrives ends by its
    20 ms limit with DF_ETIMEOUT; the network then still computes correctly."""
    from paper_1611_03226_b300 import _lib as L
    w = synth.dpd_tiny()
    net, ids = EN.dpd_fused(Net, w.h, w.orders, w.block_len, 0, 4)
    assert net.selftest_wait_timeout(20_000_000) == L.DF_ETIMEOUT
    x = w.blocks(0, 3)
    net.push(ids["ctrl"], np.ascontiguousarray(w.masks[:3]))
    net.push(ids["data"], x)
    assert net.run(-1, L.DF_RUN_PERSISTENT) == 3
    ye = net.pop(ids["sink"], dtype=np.complex64).reshape(3, -1)
    net.close()
    onet, oi = ON.dpd_fused(w.h, w.orders, w.block_len, 0, 4)
    onet.push(oi["ctrl"], ON.as_tokens_ctrl(w.masks[:3]))
    onet.push(oi["data"], ON.as_tokens_blocks(x))
    onet.run(-1)
    check_blocks(np.array(onet.pop(oi["sink"])), ye)
