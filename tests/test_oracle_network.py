"""Pins for the dataflow interpreter (Sec. 2.2 semantics): conservation, FIFO
order, validation, and Kahn determinism under every firing order."""
import numpy as np
import pytest

from oracle import actors as A
from oracle.network import FullError, Network, NetworkError, Sink, Source


def seq_tokens(start, n, nbytes):
    """Tokens carrying their sequence number in the first 4 bytes."""
    out = []
    for i in range(start, start + n):
        t = np.zeros(nbytes, np.uint8)
        t[:4] = np.frombuffer(np.uint32(i).tobytes(), np.uint8)
        out.append(t)
    return out


def chain(rates, caps, delays=None, nbytes=4, record=False):
    """source -> copy -> copy ... -> sink; channel i has (rate_i, cap_i, delay_i).
    Token sizes keep bytes per firing equal across each copy actor."""
    net = Network(record)
    src = net.add_actor(Source())
    prev, prev_port = src, 0
    ids = []
    n = len(rates)
    delays = delays or [0] * n
    # choose token sizes so that copy k moves rates[k]*S_k == rates[k+1]*S_{k+1} bytes
    sizes = [nbytes]
    for k in range(1, n):
        tot = rates[k - 1] * sizes[-1]
        assert tot % rates[k] == 0
        sizes.append(tot // rates[k])
    for k in range(n):
        dst = net.add_actor(Sink() if k == n - 1 else A.Copy())
        init = [np.full(sizes[k], 0xEE, np.uint8) for _ in range(delays[k])]
        ids.append(net.connect(prev, prev_port, dst, 0, rates[k], caps[k], init, sizes[k]))
        prev, prev_port = dst, 0
    net.finalize()
    return net, src, prev, ids


def test_conservation_and_order():
    rng = np.random.default_rng(0)
    net, src, sink, chs = chain([1, 2, 1, 3], [3, 5, 4, 7], nbytes=6)
    pushed, popped = 0, []
    for _ in range(40):
        n = int(rng.integers(0, 4))
        free = net.channels[chs[0]].free
        if n <= free:
            net.push(src, seq_tokens(pushed, n, 6))
            pushed += n
        net.run(int(rng.integers(0, 3)))
        popped += net.pop(sink, int(rng.integers(0, 5)))
        for cid in chs:                       # P5: produced + d = consumed + occupancy
            ch = net.channels[cid]
            assert ch.produced + ch.n_initial == ch.consumed + ch.occupancy
            assert 0 <= ch.occupancy <= ch.capacity
    net.run(-1)
    popped += net.pop(sink)
    data = np.concatenate(popped) if popped else np.zeros(0, np.uint8)
    # P6: bytes arrive in order; every 6-byte source token reappears intact
    n_full = len(data) // 6
    seq = [int(np.frombuffer(data[6 * i:6 * i + 4].tobytes(), np.uint32)[0]) for i in range(n_full)]
    assert seq == list(range(n_full))


def test_delay_tokens_come_first():
    net, src, sink, chs = chain([1, 1], [4, 4], delays=[0, 2], nbytes=4)
    net.push(src, seq_tokens(0, 3, 4))
    net.run(-1)
    out = net.pop(sink)
    assert [bytes(t) for t in out[:2]] == [b"\xee" * 4] * 2
    assert [int(np.frombuffer(t[:4].tobytes(), np.uint32)[0]) for t in out[2:]] == [0, 1]


def test_push_all_or_nothing():
    net, src, sink, chs = chain([1], [3])
    net.push(src, seq_tokens(0, 2, 4))
    with pytest.raises(FullError):
        net.push(src, seq_tokens(2, 2, 4))
    assert net.channels[chs[0]].occupancy == 2


def test_validation():
    net = Network()
    s = net.add_actor(Source())
    d = net.add_actor(A.DpdPoly((1,)))
    with pytest.raises(NetworkError):
        net.connect(s, 0, d, 0, 2, 4, token_bytes=4)          # control rate must be 1
    with pytest.raises(NetworkError):
        net.connect(s, 0, d, 0, 1, 4, [np.uint32(1)], 4)      # no delay on control
    with pytest.raises(NetworkError):
        net.connect(s, 0, d, 1, 3, 2, token_bytes=8)          # capacity < rate
    with pytest.raises(NetworkError):
        net.connect(s, 0, d, 1, 0, 2, token_bytes=8)          # rate 0
    net.connect(s, 0, d, 1, 1, 2, token_bytes=8)
    with pytest.raises(NetworkError):
        net.connect(s, 0, d, 0, 1, 2, token_bytes=4)          # port already connected


class Route(A.Actor):
    """Dynamic test actor: in 0 control, in 1 data; copies the data token to each
    output whose bit is set (a Poly with identity branches)."""
    dynamic = True

    def port_rates(self, ctrl, in_r, out_r):
        return dict(in_r), {k: (r if (int(ctrl) >> k) & 1 else 0) for k, r in out_r.items()}

    def fire(self, ctrl, inputs):
        return {k: [t.copy() for t in inputs[1]] for k in range(8) if (int(ctrl) >> k) & 1}


class Merge(A.Actor):
    """Dynamic test actor: in 0 control, in k+1 branch k; output = XOR of active inputs
    (zero token when none is active)."""
    dynamic = True

    def __init__(self, nbytes, r=1):
        self.nbytes, self.r = nbytes, r

    def port_rates(self, ctrl, in_r, out_r):
        return {p: (r if (int(ctrl) >> (p - 1)) & 1 else 0) for p, r in in_r.items()}, dict(out_r)

    def fire(self, ctrl, inputs):
        out = []
        for i in range(self.r):
            acc = np.zeros(self.nbytes, np.uint8)
            for p, toks in inputs.items():
                acc ^= toks[i]
            out.append(acc)
        return {0: out}


def diamond(cap_branch=2, cap=3, record=True, delay=0):
    """ctrl & data sources -> Route -> (copy | copy) -> Merge -> sink."""
    net = Network(record)
    c = net.add_actor(Source())
    x = net.add_actor(Source())
    r = net.add_actor(Route())
    b0 = net.add_actor(A.Copy())
    b1 = net.add_actor(A.Copy())
    m = net.add_actor(Merge(2))
    k = net.add_actor(Sink())
    net.connect(c, 0, r, 0, 1, cap, token_bytes=4)
    net.connect(c, 1, m, 0, 1, cap, token_bytes=4)
    net.connect(x, 0, r, 1, 1, cap, [np.array([9, 9], np.uint8)] * delay, 2)
    net.connect(r, 0, b0, 0, 1, cap_branch, token_bytes=2)
    net.connect(r, 1, b1, 0, 1, cap_branch, token_bytes=2)
    net.connect(b0, 0, m, 1, 1, cap_branch, token_bytes=2)
    net.connect(b1, 0, m, 2, 1, cap_branch, token_bytes=2)
    net.connect(m, 0, k, 0, 1, cap + 3, token_bytes=2)
    net.finalize()
    return net, c, x, k


def _load(net, c, x, masks, n):
    net.push(c, [np.uint32(v) for v in masks])
    net.push(x, [np.array([i + 1, 2 * i + 1], np.uint8) for i in range(n)])


def _histories(net):
    return [[bytes(np.asarray(t).tobytes()) for t in ch.history] for ch in net.channels]


@pytest.mark.parametrize("masks", [[1, 3, 2], [2, 2, 3], [0, 3, 1]])
def test_kahn_determinism(masks):
    """P7: sweep, random-order, threaded and every interleaving reach one quiescent state."""
    ref, c, x, k = diamond()
    _load(ref, c, x, masks, 3)
    ref.run(-1)
    want = _histories(ref)
    for seed in range(6):
        net, c, x, k = diamond()
        _load(net, c, x, masks, 3)
        net.run_random(np.random.default_rng(seed))
        assert _histories(net) == want
    net, c, x, k = diamond()
    _load(net, c, x, masks, 3)
    net.run_threaded()
    assert _histories(net) == want
    net, c, x, k = diamond()
    _load(net, c, x, masks, 3)
    finals, n_states = net.enumerate_quiescent()
    assert len(finals) == 1 and n_states > 5
    # the expected output, computed by hand from the actor definitions
    data = [np.array([i + 1, 2 * i + 1], np.uint8) for i in range(3)]
    exp = []
    for m, d in zip(masks, data):
        acc = np.zeros(2, np.uint8)
        for b in range(2):
            if (m >> b) & 1:
                acc ^= d
        exp.append(acc.tobytes())
    assert want[-1] == exp


def test_deadlock_quiescent_without_delay():
    """A feedback loop without an initial token never fires (quiescent at once)."""
    net = Network()
    a = net.add_actor(A.Copy())
    b = net.add_actor(A.Copy())
    net.connect(a, 0, b, 0, 1, 2, token_bytes=1)
    net.connect(b, 0, a, 0, 1, 2, token_bytes=1)
    net.finalize()
    assert net.run(-1) == 0
    # with one delay token the loop circulates it forever; bounded steps still work
    net = Network()
    a = net.add_actor(A.Copy())
    b = net.add_actor(A.Copy())
    net.connect(a, 0, b, 0, 1, 2, token_bytes=1)
    net.connect(b, 0, a, 0, 1, 2, [np.array([7], np.uint8)], 1)
    net.finalize()
    assert net.run(3) == 6
