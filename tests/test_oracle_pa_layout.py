"""Pins for the power-amplifier model and for Eq. 1 / Fig. 2."""
import copy
import json
import os

import pytest

import numpy as np

from oracle import pa, paper_layout as PL

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_saleh_small_signal_and_peak_p12():
    aa, ba, ap, bp = 2.1587, 1.1517, 4.0033, 9.1040
    r = np.array([1e-6, 1e-4])
    np.testing.assert_allclose(pa.saleh_am(r, aa, ba) / r, aa, rtol=1e-7)   # A(r) ~ alpha r
    np.testing.assert_allclose(pa.saleh_pm(r, ap, bp) / r ** 2, ap, rtol=1e-7)
    grid = np.linspace(0.01, 3, 300001)
    rpk = grid[np.argmax(pa.saleh_am(grid, aa, ba))]
    assert abs(rpk - 1 / np.sqrt(ba)) < 1e-4                                # peak at 1/sqrt(beta)
    assert abs(pa.saleh_am(1 / np.sqrt(ba), aa, ba) - aa / (2 * np.sqrt(ba))) < 1e-12
    x = np.array([1e-5 + 0j, 0, 0, 0])
    y = pa.pa(x)
    np.testing.assert_allclose(y[:3] / 1e-5, aa * np.array([1.0, 0.1, -0.05]), rtol=1e-6)
    assert abs(pa.small_signal_gain() - aa * 1.05) < 1e-12


def test_eq1_reproduces_table1_p13():
    g = json.load(open(os.path.join(GOLD, "table1_buffer_memory.json")))
    S, r = g["motion_token_bytes"], g["motion_gpu_rate"]
    n_delay = g["motion_channels_with_delay"]
    n_plain = len(g["motion_channels"]) - n_delay
    total = n_plain * PL.eq1_capacity_bytes(S, r, False) + n_delay * PL.eq1_capacity_bytes(S, r, True)
    assert total == 3456000
    assert round(total / 1e6, 2) == g["prop_heterog_MB"]


def test_fig2_access_pattern():
    g = json.load(open(os.path.join(GOLD, "fig2_access_pattern.json")))
    r = g["rate"]
    assert PL.eq1_capacity_tokens(r, True) == g["slots"]
    assert [PL.write_slots(k, r) for k in range(4)] == g["writes"]
    assert [PL.read_slots(k, r) for k in range(4)] == g["reads"]


def test_triple_buffer_is_a_fifo():
    """Alternating writes and reads through the Fig. 2 layout deliver D, then the
    written tokens in order (the slot 3r -> 0 copy carries the overlap)."""
    for r in (1, 2, 4, 5):
        tb = PL.TripleBuffer(r, "D")
        got, nxt = [], 0
        for _ in range(9):
            tb.write(list(range(nxt, nxt + r)))
            nxt += r
            got += tb.read()
        assert got == ["D"] + list(range(9 * r - 1))


def _orders_deliver_fifo(make, r, bound, depth):
    """Depth-first over every order of window writes and reads in which a write
    is allowed iff unread + r <= bound and a read iff r tokens are unread; True
    iff every read returns the next r tokens of the stream."""
    def dfs(buf, nxt_w, nxt_r, d):
        if d == 0:
            return True
        ok = True
        if buf.unread() + r <= bound:
            b = copy.deepcopy(buf)
            b.write(list(range(nxt_w, nxt_w + r)))
            ok = ok and dfs(b, nxt_w + r, nxt_r, d - 1)
        if ok and buf.unread() >= r:
            b = copy.deepcopy(buf)
            got = b.read()
            ok = got == list(range(nxt_r, nxt_r + r)) and dfs(b, nxt_w, nxt_r + r, d - 1)
        return ok
    buf = make()
    first_read = -1 if isinstance(buf, PL.TripleBuffer) else 0   # the delay token is token -1
    return dfs(buf, 0, first_read, depth)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_eq1_unread_capacity_is_the_exact_bound(r):
    """The reading of Fig. 2: a delay buffer of 3r + 1 slots holds at most 3r
    unread tokens, a double buffer 2r; one more window breaks FIFO order."""
    for make, delay in ((lambda: PL.TripleBuffer(r, -1), True), (lambda: PL.DoubleBuffer(r), False)):
        cap = PL.eq1_unread_capacity(r, delay)
        assert cap + (1 if delay else 0) == PL.eq1_capacity_tokens(r, delay)
        assert _orders_deliver_fifo(make, r, cap, 12)
        assert not _orders_deliver_fifo(make, r, cap + r, 12)


def test_oracle_network_eq1_capacities_and_pipeline():
    """capacity="eq1" gives 2r unread tokens to a plain channel and 3r to a delay
    channel; the paper's pipeline built that way still computes the motion maps,
    and more than one delay token is refused."""
    import synth
    from oracle import motion_paper as MP
    from oracle import nets as ON
    from oracle.network import Network, NetworkError, Sink, Source
    from oracle import actors as A
    for rate in (1, 4):
        net, ids = ON.motion_paper(16, 32, "eq1", rate)
        caps = [net.channels[ids[k]].capacity for k in ("ch_in", "ch_cur", "ch_prev", "ch_map", "ch_out")]
        assert caps == [2 * rate, 2 * rate, 3 * rate, 2 * rate, 2 * rate]
        f = synth.uniform_frames(4 * rate, 16, 32)
        got = []
        for i in range(0, len(f), rate):
            net.push(ids["src"], list(f[i:i + rate]))
            net.run(-1)
            got += net.pop(ids["sink"])
        assert np.array_equal(np.array(got), MP.pipeline(f))
    net = Network()
    a, c = net.add_actor(Source()), net.add_actor(A.Copy())
    with pytest.raises(NetworkError):
        net.connect(a, 0, c, 0, 2, "eq1", [b"xx", b"yy"], 2)
