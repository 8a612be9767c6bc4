"""Pins for the predistortion oracle (Sec. 4.2 network, float64).

Each expected value below is computed by a route that shares nothing with the
oracle's arithmetic: numpy.convolve / scipy.signal.lfilter for the FIRs,
np.abs(x)**(o-1) for the branch nonlinearity, and central finite differences
for the adjoint."""
import numpy as np
import pytest
from scipy.signal import lfilter

from oracle import dpd as D
from oracle import nets

import synth


def run_stream(net, ids, masks, blocks, push_chunk, rng=None):
    """Push control and data in chunks, run, pop; returns the concatenated output."""
    out = []
    i = 0
    n = len(masks)
    while i < n or net.channels[ids["ch_out"]].occupancy or any(
            net.enabled(a) for a in range(len(net.actors))):
        k = min(push_chunk, n - i, net.channels[ids["ch_data"]].free, net.channels[0].free)
        if k > 0:
            net.push(ids["ctrl"], nets.as_tokens_ctrl(masks[i:i + k]))
            net.push(ids["data"], nets.as_tokens_blocks(blocks[i:i + k]))
            i += k
        net.run(1 if rng is None else int(rng.integers(1, 3)))
        out += net.pop(ids["sink"])
        if i >= n and not any(net.enabled(a) for a in range(len(net.actors))):
            out += net.pop(ids["sink"])
            break
    return np.concatenate(out) if out else np.zeros(0, np.complex128)


def delayed(blocks, d):
    L = blocks.shape[1]
    s = np.concatenate([np.zeros(d * L, np.complex128), blocks.reshape(-1).astype(np.complex128)])
    return s[:blocks.size]


def small_workload(n_blocks=12, L=64, K=4, M=10, seed=5):
    rng = np.random.default_rng(seed)
    x = (rng.normal(0, 0.3, (n_blocks, L)) + 1j * rng.normal(0, 0.3, (n_blocks, L))).astype(np.complex64)
    h = (rng.normal(0, 0.1, (K, M)) + 1j * rng.normal(0, 0.1, (K, M))).astype(np.complex64)
    return rng, x, h


def test_identity_predistorter_p1():
    rng, x, _ = small_workload()
    K, M = 4, 10
    h = np.zeros((K, M), np.complex64)
    h[0, 0] = 1
    masks = (rng.integers(0, 16, size=len(x)) | 1).astype(np.uint32)
    net, ids = nets.dpd_fused(h, (1, 3, 5, 7), x.shape[1], delay=2, capacity=4)
    y = run_stream(net, ids, masks, x, push_chunk=2)
    assert len(y) == x.size
    np.testing.assert_array_equal(y, delayed(x, 2))        # exact, incl. the 2 zero blocks
    for cid in range(len(net.channels)):
        p, c, o = net.counters(cid)
        assert p + net.channels[cid].n_initial == c + o


def test_single_branch_is_closed_form_fir_p2():
    rng, x, h = small_workload()
    masks = np.ones(len(x), np.uint32)
    net, ids = nets.dpd_fused(h, (1, 3, 5, 7), x.shape[1], delay=1, capacity=3)
    y = run_stream(net, ids, masks, x, push_chunk=1)
    s = delayed(x, 1)
    want = np.convolve(s, h[0].astype(np.complex128))[:len(s)]
    assert D.rel_l2(y, want) < 1e-13


def _branch(x, o):
    return np.abs(x.astype(np.complex128)) ** (o - 1) * x.astype(np.complex128)


def test_all_branches_active_p3():
    rng, x, h = small_workload()
    orders = (1, 3, 5, 7)
    masks = np.full(len(x), 15, np.uint32)
    net, ids = nets.dpd_fused(h, orders, x.shape[1], delay=0, capacity=5)
    y = run_stream(net, ids, masks, x, push_chunk=3)
    s = x.reshape(-1)
    want = sum(np.convolve(_branch(s, o), h[k].astype(np.complex128))[:len(s)]
               for k, o in enumerate(orders))
    assert D.rel_l2(y, want) < 1e-13


def restatement(x_blocks, h, orders, masks, d):
    """Per branch: concatenate the branch signal of the blocks where it is active,
    filter the whole concatenation, cut it back into blocks, add (P4)."""
    L = x_blocks.shape[1]
    blocks = [np.zeros(L, np.complex128)] * d + [b.astype(np.complex128) for b in x_blocks]
    n = len(masks)
    out = np.zeros((n, L), np.complex128)
    for k, o in enumerate(orders):
        act = [i for i in range(n) if (int(masks[i]) >> k) & 1]
        if not act:
            continue
        z = np.concatenate([_branch(blocks[i], o) for i in act])
        yk = lfilter(h[k].astype(np.complex128), [1.0], z)
        for j, i in enumerate(act):
            out[i] += yk[j * L:(j + 1) * L]
    return out.reshape(-1)


@pytest.mark.parametrize("L,M,d", [(64, 10, 1), (3, 10, 2), (1, 4, 0), (17, 16, 2)])
def test_random_masks_restatement_p4(L, M, d):
    rng = np.random.default_rng(L * 100 + M)
    n = 20
    orders = tuple(range(1, 16, 2))
    x = (rng.normal(0, 0.3, (n, L)) + 1j * rng.normal(0, 0.3, (n, L))).astype(np.complex64)
    h = (rng.normal(0, 0.1, (8, M)) + 1j * rng.normal(0, 0.1, (8, M))).astype(np.complex64)
    masks = rng.integers(0, 256, size=n).astype(np.uint32)
    net, ids = nets.dpd_fused(h, orders, L, delay=d, capacity=d + 3)
    y = run_stream(net, ids, masks, x, push_chunk=2, rng=rng)
    want = restatement(x, h, orders, masks, d)[:len(y)]
    assert len(y) == (n) * L
    assert D.rel_l2(y, want) < 1e-12


def test_expanded_network_equals_fused():
    """The literal Poly -> FIR_k -> Adder network (small branch FIFOs, many sweeps)
    produces exactly the fused actor's stream (Kahn determinism + composition)."""
    w = synth.dpd_tiny()
    x = w.blocks(0, 16)[:, :256]
    masks = w.masks[:16]
    f, fi = nets.dpd_fused(w.h, w.orders, 256, delay=1, capacity=6)
    e, ei = nets.dpd_expanded(w.h, w.orders, 256, delay=1, capacity=6, branch_capacity=2)
    yf = run_stream(f, fi, masks, x, push_chunk=4)
    ye = run_stream(e, ei, masks, x, push_chunk=4)
    np.testing.assert_array_equal(yf, ye)


def test_stateless_stream_matches_network():
    rng, x, h = small_workload(n_blocks=1, L=300)
    orders = (1, 3, 5, 7)
    net, ids = nets.dpd_fused(h, orders, 300, delay=0, capacity=2)
    y = run_stream(net, ids, np.array([15], np.uint32), x, push_chunk=1)
    np.testing.assert_array_equal(y, D.dpd_stream(x[0], h, orders))


def test_adjoint_against_finite_differences_p11():
    rng = np.random.default_rng(11)
    N, K, M = 40, 3, 4
    orders = (1, 3, 5)
    x = rng.normal(0, 0.4, N) + 1j * rng.normal(0, 0.4, N)
    h = rng.normal(0, 0.3, (K, M)) + 1j * rng.normal(0, 0.3, (K, M))
    W = rng.normal(size=N) + 1j * rng.normal(size=N)

    def loss(x, h):       # real loss with dL/dRe(y) + i dL/dIm(y) = W
        return float(np.real(np.sum(np.conj(W) * D.dpd_stream(x, h, orders))))

    gx, gh = D.dpd_stream_backward(x, h, orders, W)
    eps = 1e-6
    for k in range(K):
        for m in range(M):
            for unit in (1.0, 1j):
                hp, hm = h.copy(), h.copy()
                hp[k, m] += eps * unit
                hm[k, m] -= eps * unit
                fd = (loss(x, hp) - loss(x, hm)) / (2 * eps)
                an = gh[k, m].real if unit == 1.0 else gh[k, m].imag
                assert abs(fd - an) < 1e-8 * max(1.0, abs(an))
    for j in list(range(0, N, 3)) + [N - 1]:
        for unit in (1.0, 1j):
            xp, xm = x.copy(), x.copy()
            xp[j] += eps * unit
            xm[j] -= eps * unit
            fd = (loss(xp, h) - loss(xm, h)) / (2 * eps)
            an = gx[j].real if unit == 1.0 else gx[j].imag
            assert abs(fd - an) < 1e-8 * max(1.0, abs(an))


def test_psi_orders():
    x = np.array([0.3 - 0.4j, 2.0 + 0j, 0j])
    np.testing.assert_allclose(D.psi(x, 1), x)
    np.testing.assert_allclose(D.psi(x, 3), np.abs(x) ** 2 * x, rtol=1e-15)
    np.testing.assert_allclose(D.psi(x, 15), np.abs(x) ** 14 * x, rtol=1e-13)
    with pytest.raises(ValueError):
        D.psi(x, 2)
