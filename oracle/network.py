"""Sequential interpreter for the dataflow model of Sec. 2.2 (oracle; test infrastructure).

Model (Sec. 2.2, Sec. 3.1, Sec. 3.2):

* A network is a set of actors and a set of FIFO channels.  A channel joins
  exactly one output port to exactly one input port and preserves order.
* Each channel f has a token rate r > 0; the ports at both ends adopt it.
  Reads and writes block until enough tokens / free slots exist.
* A static actor always uses its port rates.  A dynamic actor has one control
  input port of rate 1; per firing it reads one control token, and the control
  function fixes each regular port's rate to 0 or r for that firing.
* Channels not attached to a control port may hold initial (delay) tokens.
  The paper allows 0 or 1 and notes the generalisation to more; this
  interpreter accepts any count below the capacity.
* Capacity is chosen by the user, or, with capacity="eq1", fixed as the paper
  does by Eq. 1: 2r unread tokens without a delay token, 3r with one (the
  reading of Fig. 2 in :mod:`oracle.paper_layout`).

Reading adopted for bounded steps (the paper runs one thread per actor and has
no notion of a step): ``run(n)`` performs n sweeps; a sweep visits the actors
in the order they were added and fires each one repeatedly while it is
enabled.  ``run(-1)`` sweeps until a sweep fires nothing.  Final channel
histories are independent of the firing order (Kahn determinism); the
random-order scheduler, the threaded runner and the brute-force enumeration
below exist to test exactly that.

A variable-rate output port (beyond the paper's two rates, cf. Sec. 5) has a
maximum rate r_max: the actor is enabled only if r_max slots are free, and it
produces between 0 and r_max tokens.
"""
from __future__ import annotations

import copy
import threading
from collections import deque

import numpy as np

from . import paper_layout


class NetworkError(Exception):
    pass


class FullError(NetworkError):
    pass


class Channel:
    """Bounded order-preserving FIFO (Sec. 2.2, Sec. 3.2)."""

    def __init__(self, cid, src, src_port, dst, dst_port, token_bytes, rate,
                 capacity, initial, record_history=False):
        self.cid = cid
        self.src, self.src_port = src, src_port
        self.dst, self.dst_port = dst, dst_port
        self.token_bytes = token_bytes
        self.rate = rate
        self.capacity = capacity
        self.q = deque(initial)
        self.n_initial = len(initial)
        self.produced = 0          # tokens written after start (excludes initial tokens)
        self.consumed = 0          # tokens read
        self.reserved = 0          # slots promised to an in-flight firing (threaded runner)
        self.history = list(initial) if record_history else None

    @property
    def occupancy(self) -> int:
        return len(self.q)

    @property
    def free(self) -> int:
        return self.capacity - len(self.q) - self.reserved

    def write(self, toks):
        if len(toks) > self.capacity - len(self.q):
            raise FullError(f"channel {self.cid}: write of {len(toks)} exceeds free space")
        self.q.extend(toks)
        self.produced += len(toks)
        if self.history is not None:
            self.history.extend(toks)

    def read(self, n):
        out = [self.q.popleft() for _ in range(n)]
        self.consumed += n
        return out


class Actor:
    """Actor base (Sec. 3.1): ``fire`` is mandatory, ``control`` is for dynamic actors.

    Subclasses set ``dynamic`` and implement ``port_rates(ctrl, in_r, out_r)``
    returning the per-port rates for one firing, and ``fire(ctrl, inputs)``
    returning ``{out_port: [tokens]}``.  For dynamic actors input port 0 is the
    control port; ``inputs`` never contains it.
    """
    dynamic = False
    host_endpoint = False          # sources / sinks are driven by push / pop
    variable_out_ports: tuple = ()

    def port_rates(self, ctrl, in_r, out_r):
        return dict(in_r), dict(out_r)

    def fire(self, ctrl, inputs):
        raise NotImplementedError

    def validate(self, in_ch, out_ch):
        pass


class Source(Actor):
    """Host push endpoint; every pushed token is written to all output channels."""
    host_endpoint = True


class Sink(Actor):
    """Host pop endpoint with one input channel."""
    host_endpoint = True


class Network:
    def __init__(self, record_history=False):
        self.actors = []
        self.channels = []
        self.in_ch = []            # per actor: {port: Channel}
        self.out_ch = []
        self.finalized = False
        self.record_history = record_history

    # ---- construction (mirrors net_create / actor_add / channel_connect) ----
    def add_actor(self, actor: Actor) -> int:
        if self.finalized:
            raise NetworkError("network is finalized")
        self.actors.append(actor)
        self.in_ch.append({})
        self.out_ch.append({})
        return len(self.actors) - 1

    def connect(self, src, src_port, dst, dst_port, rate, capacity, initial=(),
                token_bytes=None) -> int:
        if self.finalized:
            raise NetworkError("network is finalized")
        if rate <= 0:
            raise NetworkError("token rate must be positive (Sec. 2.2)")
        if src_port in self.out_ch[src] or dst_port in self.in_ch[dst]:
            raise NetworkError("a port connects to exactly one channel (Sec. 3.2)")
        initial = list(initial)
        if capacity == "eq1":
            if len(initial) > 1:
                raise NetworkError("Eq. 1 covers at most one delay token (Sec. 3.2)")
            capacity = paper_layout.eq1_unread_capacity(rate, len(initial) == 1)
        if capacity < len(initial) + rate:
            raise NetworkError("capacity must hold the initial tokens plus one firing")
        dst_actor = self.actors[dst]
        if dst_actor.dynamic and dst_port == 0:
            if rate != 1 or initial:
                raise NetworkError("control channel: rate 1, no initial tokens (Sec. 2.2)")
        ch = Channel(len(self.channels), src, src_port, dst, dst_port, token_bytes, rate,
                     capacity, initial, self.record_history)
        self.channels.append(ch)
        self.out_ch[src][src_port] = ch
        self.in_ch[dst][dst_port] = ch
        return ch.cid

    def finalize(self):
        for a, actor in enumerate(self.actors):
            for ports in (self.in_ch[a], self.out_ch[a]):
                if ports and sorted(ports) != list(range(len(ports))):
                    raise NetworkError(f"actor {a}: ports must be numbered 0..n-1")
            if isinstance(actor, Sink) and len(self.in_ch[a]) != 1:
                raise NetworkError("a sink has exactly one input")
            actor.validate(self.in_ch[a], self.out_ch[a])
        self.finalized = True

    # ---- host endpoints ----
    def push(self, src, tokens):
        """All-or-nothing broadcast of ``tokens`` to every output channel of a source."""
        tokens = list(tokens)
        chans = list(self.out_ch[src].values())
        if any(ch.free < len(tokens) for ch in chans):
            raise FullError("push: not enough free space")
        for ch in chans:
            ch.write([copy.copy(t) for t in tokens])
        return len(tokens)

    def pop(self, sink, max_tokens=None):
        ch = self.in_ch[sink][0]
        n = ch.occupancy if max_tokens is None else min(max_tokens, ch.occupancy)
        return ch.read(n)

    def counters(self, cid):
        ch = self.channels[cid]
        return ch.produced, ch.consumed, ch.occupancy

    # ---- firing rule (Sec. 2.2) ----
    def _rates(self, a):
        actor = self.actors[a]
        ins, outs = self.in_ch[a], self.out_ch[a]
        ctrl = None
        if actor.dynamic:
            cch = ins[0]
            if not cch.q:
                return None
            ctrl = cch.q[0]
        in_r = {p: ch.rate for p, ch in ins.items() if not (actor.dynamic and p == 0)}
        out_r = {p: ch.rate for p, ch in outs.items()}
        rin, rout = actor.port_rates(ctrl, in_r, out_r)
        return ctrl, rin, rout

    def enabled(self, a) -> bool:
        actor = self.actors[a]
        if actor.host_endpoint:
            return False
        r = self._rates(a)
        if r is None:
            return False
        _, rin, rout = r
        ins, outs = self.in_ch[a], self.out_ch[a]
        if any(k and ins[p].occupancy < k for p, k in rin.items()):
            return False
        if any(k and outs[p].free < k for p, k in rout.items()):
            return False
        return True

    def _take(self, a):
        """Consume the control token and input windows of one enabled firing."""
        actor = self.actors[a]
        ctrl, rin, rout = self._rates(a)
        ins = self.in_ch[a]
        if actor.dynamic:
            ins[0].read(1)
        inputs = {p: ins[p].read(k) for p, k in rin.items() if k}
        return ctrl, rout, inputs

    def _give(self, a, rout, outputs):
        actor = self.actors[a]
        outs = self.out_ch[a]
        for p, k in rout.items():
            toks = outputs.get(p, [])
            if p in actor.variable_out_ports:
                if len(toks) > k:
                    raise NetworkError("variable-rate port produced more than r_max")
            elif len(toks) != k:
                raise NetworkError(f"actor {a} port {p}: produced {len(toks)} tokens, rate {k}")
            if toks:
                outs[p].write(toks)

    def fire_once(self, a):
        ctrl, rout, inputs = self._take(a)
        self._give(a, rout, self.actors[a].fire(ctrl, inputs))

    # ---- schedulers ----
    def sweep(self) -> int:
        fired = 0
        for a in range(len(self.actors)):
            while self.enabled(a):
                self.fire_once(a)
                fired += 1
        return fired

    def run(self, n_steps=-1) -> int:
        if not self.finalized:
            raise NetworkError("finalize first")
        total, step = 0, 0
        while n_steps < 0 or step < n_steps:
            f = self.sweep()
            total += f
            step += 1
            if n_steps < 0 and f == 0:
                break
        return total

    def run_random(self, rng: np.random.Generator) -> int:
        """Fire one uniformly chosen enabled actor at a time until quiescent."""
        total = 0
        while True:
            en = [a for a in range(len(self.actors)) if self.enabled(a)]
            if not en:
                return total
            self.fire_once(int(rng.choice(en)))
            total += 1

    def run_threaded(self, timeout=30.0) -> int:
        """One thread per actor with blocking channel access (Sec. 3.3).

        Inputs are taken and output space reserved under one lock, the actor body
        runs outside it, and outputs are written back under the lock.  The run
        ends when every thread is blocked and no firing is in flight.
        """
        cv = threading.Condition()
        state = {"waiting": 0, "busy": 0, "done": False, "fired": 0, "error": None}
        workers = [a for a in range(len(self.actors)) if not self.actors[a].host_endpoint]

        def body(a):
            actor = self.actors[a]
            while True:
                with cv:
                    while not state["done"] and not self.enabled(a):
                        state["waiting"] += 1
                        if (state["waiting"] == len(workers) and state["busy"] == 0
                                and not any(self.enabled(w) for w in workers)):
                            state["done"] = True
                            cv.notify_all()
                        else:
                            if not cv.wait(timeout):
                                state["error"] = "threaded runner timed out"
                                state["done"] = True
                                cv.notify_all()
                        state["waiting"] -= 1
                    if state["done"]:
                        return
                    ctrl, rout, inputs = self._take(a)
                    for p, k in rout.items():
                        self.out_ch[a][p].reserved += k
                    state["busy"] += 1
                try:
                    outputs = actor.fire(ctrl, inputs)
                except Exception as e:          # surfaced to the caller below
                    outputs = None
                    err = e
                with cv:
                    for p, k in rout.items():
                        self.out_ch[a][p].reserved -= k
                    if outputs is None:
                        state["error"] = repr(err)
                        state["done"] = True
                    else:
                        self._give(a, rout, outputs)
                        state["fired"] += 1
                    state["busy"] -= 1
                    cv.notify_all()

        threads = [threading.Thread(target=body, args=(a,), daemon=True) for a in workers]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout * 4)
        if state["error"]:
            raise NetworkError(state["error"])
        return state["fired"]

    # ---- brute force (tiny networks only) ----
    def _state_key(self):
        chans = tuple(tuple(_key(t) for t in ch.q) for ch in self.channels)
        acts = tuple(_key(getattr(a, "state_key", lambda: None)()) for a in self.actors)
        return chans, acts

    def enumerate_quiescent(self, limit=200000):
        """All distinct quiescent states reachable by any interleaving of single firings."""
        seen, finals, stack = set(), set(), [copy.deepcopy(self)]
        while stack:
            net = stack.pop()
            key = net._state_key()
            if key in seen:
                continue
            seen.add(key)
            if len(seen) > limit:
                raise NetworkError("state space too large")
            en = [a for a in range(len(net.actors)) if net.enabled(a)]
            if not en:
                finals.add(key)
            for a in en:
                nxt = copy.deepcopy(net)
                nxt.fire_once(a)
                stack.append(nxt)
        return finals, len(seen)


def _key(t):
    if isinstance(t, np.ndarray):
        return (t.dtype.str, t.shape, t.tobytes())
    if isinstance(t, (list, tuple)):
        return tuple(_key(x) for x in t)
    if isinstance(t, np.generic):
        return t.item()
    return t
