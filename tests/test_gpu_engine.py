"""Engine semantics on the GPU: multirate copy chains and diamonds step by step
against the oracle interpreter, and the C-ABI error paths."""
import numpy as np
import pytest

from oracle import actors as A
from oracle.network import Network, Sink, Source

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1611_03226_b300 as P
    return P


def build_chain(P, rates, caps, sizes, delays):
    """source -> copy -> ... -> sink on both sides; returns (onet, enet, src, sink, chans)."""
    onet, enet = Network(), P.Net()
    o_prev, e_prev = onet.add_actor(Source()), enet.add_source()
    chans = []
    n = len(rates)
    for k in range(n):
        last = k == n - 1
        od = onet.add_actor(Sink() if last else A.Copy())
        ed = enet.add_sink() if last else enet.add_copy()
        init = [np.full(sizes[k], 0x5A + k, np.uint8) for _ in range(delays[k])]
        oc = onet.connect(o_prev, 0, od, 0, rates[k], caps[k], init, sizes[k])
        ec = enet.connect(e_prev, 0, ed, 0, sizes[k], rates[k], caps[k], delays[k],
                          np.concatenate(init) if init else None)
        chans.append((oc, ec))
        o_prev, e_prev = od, ed
    onet.finalize()
    enet.finalize()
    return onet, enet, 0, o_prev, e_prev, chans


@pytest.mark.parametrize("rates,caps,sizes,delays", [
    ([1, 2, 1, 3], [3, 5, 4, 7], [6, 3, 6, 2], [0, 1, 0, 2]),
    ([4, 1, 2], [9, 3, 5], [16, 64, 32], [1, 0, 1]),
    ([3, 5], [7, 11], [5, 3], [2, 0]),
])
@pytest.mark.parametrize("persistent", [False, True])
def test_copy_chain_step_by_step(P, rates, caps, sizes, delays, persistent):
    from paper_1611_03226_b300 import _lib as L
    flags = L.DF_RUN_PERSISTENT if persistent else 0
    onet, enet, src, osink, esink, chans = build_chain(P, rates, caps, sizes, delays)
    rng = np.random.default_rng(sum(rates))
    seq = 0
    got_o, got_e = [], []
    for it in range(30):
        free = onet.channels[chans[0][0]].free
        k = int(rng.integers(0, 4))
        if 0 < k <= free:
            toks = [(np.arange((seq + j) * sizes[0], (seq + j + 1) * sizes[0]) % 251).astype(np.uint8)
                    for j in range(k)]
            onet.push(src, toks)
            enet.push(src, np.concatenate(toks))
            seq += k
        steps = int(rng.integers(0, 3))
        assert onet.run(steps) == enet.run(steps, flags)
        for oc, ec in chans:
            assert onet.counters(oc) == enet.counters(ec)
        m = int(rng.integers(0, 5))
        got_o += onet.pop(osink, m)
        got_e.append(enet.pop(esink, m))
    o = np.concatenate(got_o) if got_o else np.zeros(0, np.uint8)
    np.testing.assert_array_equal(np.concatenate(got_e), o)
    enet.close()


def test_error_paths(P):
    from paper_1611_03226_b300 import _lib as L
    net = P.Net()
    s = net.add_source()
    k = net.add_sink()
    net.connect(s, 0, k, 0, 4, 1, 3)
    with pytest.raises(L.DfError) as e:
        net.push(s, np.zeros(4, np.uint8))            # not finalized yet
    assert e.value.status == L.DF_ESTATE
    with pytest.raises(L.DfError) as e:
        net.connect(s, 0, k, 0, 4, 1, 3)              # port already connected
    assert e.value.status == L.DF_EINVAL
    with pytest.raises(L.DfError) as e:
        net.run(1)
    assert e.value.status == L.DF_ESTATE
    net.finalize()
    net.push(s, np.arange(12, dtype=np.uint8))
    with pytest.raises(L.DfError) as e:
        net.push(s, np.zeros(4, np.uint8))
    assert e.value.status == L.DF_EFULL
    assert net.counters(0) == (3, 0, 3)
    np.testing.assert_array_equal(net.pop(k), np.arange(12, dtype=np.uint8))
    net.close()
    net = P.Net()
    a = net.add_source()
    d = net.add_dpd(np.ones((1, 2), np.complex64), (1,), 8)
    with pytest.raises(L.DfError) as e:
        net.connect(a, 0, d, 0, 4, 2, 4)              # control rate must be 1
    assert e.value.status == L.DF_EINVAL
    net.close()


@pytest.mark.parametrize("delay,cap,persistent", [(3, 4, False), (1, 2, False), (5, 8, True)])
def test_feedback_cycle_with_delay_tokens(P, delay, cap, persistent):
    """A cycle A -> B -> A whose only tokens are the `delay` initial tokens on the
    edge B -> A (the feedback use of initial tokens, Sec. 2.2); A also copies every
    token to a sink, which must receive the initial tokens over and over in order."""
    from paper_1611_03226_b300 import _lib as L
    flags = L.DF_RUN_PERSISTENT if persistent else 0
    tok = 12
    init = [np.arange(i * tok, (i + 1) * tok, dtype=np.uint8) for i in range(delay)]
    onet, enet = Network(), P.Net()
    oa, ob, os_ = onet.add_actor(A.Copy()), onet.add_actor(A.Copy()), onet.add_actor(Sink())
    ea, eb, es = enet.add_copy(), enet.add_copy(), enet.add_sink()
    chans = [
        (onet.connect(ob, 0, oa, 0, 1, cap, init, tok),
         enet.connect(eb, 0, ea, 0, tok, 1, cap, delay, np.concatenate(init))),
        (onet.connect(oa, 0, ob, 0, 1, cap, [], tok), enet.connect(ea, 0, eb, 0, tok, 1, cap)),
        (onet.connect(oa, 1, os_, 0, 1, 4 * delay, [], tok), enet.connect(ea, 1, es, 0, tok, 1, 4 * delay)),
    ]
    onet.finalize()
    enet.finalize()
    got = []
    for step in range(6):
        assert onet.run(1) == enet.run(1, flags)
        for oc, ec in chans:
            assert onet.counters(oc) == enet.counters(ec)
        want = np.concatenate(onet.pop(os_))
        e = enet.pop(es)
        np.testing.assert_array_equal(e, want)
        got.append(e)
    stream = np.concatenate(got).reshape(-1, tok)
    assert len(stream) == 6 * delay
    np.testing.assert_array_equal(stream, np.tile(np.concatenate(init).reshape(delay, tok), (6, 1)))
    enet.close()
