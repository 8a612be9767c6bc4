"""Actor bodies for the oracle interpreter (test infrastructure).

Predistortion network of Sec. 4.2 (Fig. 5 is lost; its structure is taken
from the text): a configuration source feeds control tokens to a dynamic Poly
actor and a dynamic Adder actor; Poly sends the nonlinear branch signal to the
FIR actor of every branch active in this firing; the Adder sums the active
branch outputs.  Control mapping (left open by Sec. 2.2 / Sec. 3.1): the
control token is a u32 bit mask, bit k = branch k active.

Motion detection (Sec. 4.1, benchmark variant): frame difference against a
one-frame-delayed copy, threshold, erosion, dilation, tile emission with a
variable number of output records per frame.
"""
from __future__ import annotations

import numpy as np

from . import dpd as D
from . import motion as MD
from . import motion_paper as MP
from .network import Actor, NetworkError


class Copy(Actor):
    """Static actor: reads r_in tokens from input 0 and writes the same bytes to
    every output, re-cut into that channel's r_out tokens (byte count must match)."""

    def validate(self, in_ch, out_ch):
        if len(in_ch) != 1 or not out_ch:
            raise NetworkError("copy: one input, >= 1 outputs")
        ci = in_ch[0]
        for ch in out_ch.values():
            if ci.token_bytes * ci.rate != ch.token_bytes * ch.rate:
                raise NetworkError("copy: bytes per firing must match on every port")
        self._outs = dict(out_ch)

    def fire(self, ctrl, inputs):
        data = np.concatenate([np.asarray(t, np.uint8).reshape(-1) for t in inputs[0]])
        out = {}
        for p, ch in self._outs.items():
            out[p] = [data[i * ch.token_bytes:(i + 1) * ch.token_bytes].copy()
                      for i in range(ch.rate)]
        return out


class DpdPoly(Actor):
    """Dynamic: in 0 = control, in 1 = data block; out k = branch k signal psi_{o_k}(x)."""
    dynamic = True

    def __init__(self, orders):
        self.orders = tuple(orders)

    def port_rates(self, ctrl, in_r, out_r):
        return dict(in_r), {k: (r if (int(ctrl) >> k) & 1 else 0) for k, r in out_r.items()}

    def fire(self, ctrl, inputs):
        x = inputs[1]
        return {k: [D.psi(b, self.orders[k]) for b in x]
                for k in D.active_branches(ctrl, len(self.orders))}


class DpdFir(Actor):
    """Static: M-tap complex FIR over the concatenation of every block it receives."""

    def __init__(self, h):
        self.h = np.asarray(h, np.complex128)
        self.hist = np.zeros(len(self.h) - 1, np.complex128)

    def fire(self, ctrl, inputs):
        out = []
        for z in inputs[0]:
            y, self.hist = D.fir(self.h, self.hist, z)
            out.append(y)
        return {0: out}

    def state_key(self):
        return self.hist.tobytes()


class DpdAdd(Actor):
    """Dynamic: in 0 = control, in k+1 = branch k; out 0 = sum of active branches
    in ascending k (an empty mask gives a zero block)."""
    dynamic = True

    def __init__(self, K, block_len):
        self.K, self.block_len = K, block_len
        self.r_out = 1

    def validate(self, in_ch, out_ch):
        self.r_out = out_ch[0].rate

    def port_rates(self, ctrl, in_r, out_r):
        return {p: (r if (int(ctrl) >> (p - 1)) & 1 else 0) for p, r in in_r.items()}, dict(out_r)

    def fire(self, ctrl, inputs):
        n = self.r_out
        out = []
        for i in range(n):
            acc = np.zeros(self.block_len, np.complex128)
            for k in D.active_branches(ctrl, self.K):
                acc = acc + inputs[k + 1][i]
            out.append(acc)
        return {0: out}


class Dpd(Actor):
    """Fused predistorter (Poly -> FIR_k -> Adder run in sequence inside one firing).

    Ports: in 0 = control (u32 mask), in 1 = data block, out 0 = output block.
    Branch k's FIR sees only the blocks in which branch k was active, exactly
    as in the expanded network.
    """
    dynamic = True

    def __init__(self, h, orders, block_len):
        h = np.asarray(h, np.complex128)
        self.orders = tuple(orders)
        self.block_len = block_len
        self.poly = DpdPoly(orders)
        self.firs = [DpdFir(h[k]) for k in range(len(orders))]
        self.add = DpdAdd(len(orders), block_len)

    def port_rates(self, ctrl, in_r, out_r):
        return dict(in_r), dict(out_r)

    def validate(self, in_ch, out_ch):
        if any(ch.rate != 1 for ch in list(in_ch.values()) + list(out_ch.values())):
            raise NetworkError("fused predistorter: all ports have rate 1")

    def fire(self, ctrl, inputs):
        zs = self.poly.fire(ctrl, {1: inputs[1]})
        ys = {k + 1: self.firs[k].fire(None, {0: zs[k]})[0] for k in zs}
        return self.add.fire(ctrl, ys)

    def state_key(self):
        return tuple(f.hist.tobytes() for f in self.firs)


class MdDiff(Actor):
    """Static: in 0 = current frame, in 1 = previous frame; out 0 = |cur - prev|."""

    def fire(self, ctrl, inputs):
        return {0: [MD.absdiff(c, p) for c, p in zip(inputs[0], inputs[1])]}


class MdThresh(Actor):
    def __init__(self, t=25):
        self.t = t

    def fire(self, ctrl, inputs):
        return {0: [MD.threshold(d, self.t) for d in inputs[0]]}


class MdErode(Actor):
    def fire(self, ctrl, inputs):
        return {0: [MD.erode3x3(b) for b in inputs[0]]}


class MdDilate(Actor):
    def fire(self, ctrl, inputs):
        return {0: [MD.dilate3x3(b) for b in inputs[0]]}


class MdTiles(Actor):
    """Static input, out 0 = records (variable rate, r_max = tiles per frame),
    out 1 = one u32 token per frame holding the number of records emitted."""
    variable_out_ports = (0,)

    def __init__(self, tile=16):
        self.tile = tile

    def fire(self, ctrl, inputs):
        recs, cnts = [], []
        for o in inputs[0]:
            r = MD.tile_records(MD.tile_counts(o, self.tile), self.tile)
            recs.extend(r[i:i + 1] for i in range(len(r)))
            cnts.append(np.array([len(r)], np.uint32))
        return {0: recs, 1: cnts}


class Md(Actor):
    """Fused motion detector: Diff -> Thresh -> Erode -> Dilate -> Tiles in one firing.

    Ports: in 0 = current frame, in 1 = previous frame; out 0 = records
    (variable rate), out 1 = per-frame record count."""
    variable_out_ports = (0,)

    def __init__(self, t=25, tile=16):
        self.t, self.tile = t, tile

    def fire(self, ctrl, inputs):
        recs, cnts = [], []
        for c, p in zip(inputs[0], inputs[1]):
            r = MD.detect(c, p, self.t, self.tile)
            recs.extend(r[i:i + 1] for i in range(len(r)))
            cnts.append(np.array([len(r)], np.uint32))
        return {0: recs, 1: cnts}


# ---- the paper's own motion pipeline (Sec. 4.1): Gauss -> Thres -> Med ----
class Gauss5(Actor):
    """Static: in 0 = frames; every output gets the filtered frames (the paper's
    Gauss feeds Thres over two channels, one with the delay token)."""

    def fire(self, ctrl, inputs):
        g = [MP.gauss5(f) for f in inputs[0]]
        return {p: [x.copy() for x in g] for p in self._outs}

    def validate(self, in_ch, out_ch):
        if len(in_ch) != 1 or not out_ch:
            raise NetworkError("gauss: one input, >= 1 outputs")
        self._outs = tuple(out_ch)


class Thres(Actor):
    """Static: in 0 = current filtered frame, in 1 = previous filtered frame; out 0 = motion map."""

    def __init__(self, t=MP.THRESHOLD):
        self.t = t

    def fire(self, ctrl, inputs):
        return {0: [MP.thres(c, p, self.t) for c, p in zip(inputs[0], inputs[1])]}


class Med5(Actor):
    """Static: in 0 = motion map; every output gets the median-filtered map."""

    def fire(self, ctrl, inputs):
        m = [MP.med5(f) for f in inputs[0]]
        return {p: [x.copy() for x in m] for p in self._outs}

    def validate(self, in_ch, out_ch):
        if len(in_ch) != 1 or not out_ch:
            raise NetworkError("med: one input, >= 1 outputs")
        self._outs = tuple(out_ch)
