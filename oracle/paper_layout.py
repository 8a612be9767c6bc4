"""Channel capacity of Eq. 1 and the delay-channel access pattern of Fig. 2
(oracle; test infrastructure).

Eq. 1: a channel with token size S and rate r holds S * 2r bytes (a double
buffer), or S * (3r + 1) bytes when it carries an initial (delay) token.

Fig. 2 (r = 4, described in Sec. 3.2): the delay token starts in slot 0; the
k-th write fills slots 1 + (k r mod 3r) ... + r - 1, the k-th read takes slots
(k r mod 3r) ... + r - 1; the write that reaches the last slot (3r) is
followed by a copy of slot 3r into slot 0, and the pattern repeats.
"""
from __future__ import annotations


def eq1_capacity_tokens(rate: int, has_delay: bool) -> int:
    return 3 * rate + 1 if has_delay else 2 * rate


def eq1_capacity_bytes(token_bytes: int, rate: int, has_delay: bool) -> int:
    return token_bytes * eq1_capacity_tokens(rate, has_delay)


def eq1_unread_capacity(rate: int, has_delay: bool) -> int:
    """Most unread tokens an Eq. 1 buffer can hold without a write landing on a
    token not yet read: all 2r slots of the double buffer; 3r of the 3r + 1
    slots of the delay buffer, because slot 0 and slot 3r hold the same token
    once the copy is made (a reading of Fig. 2, which the paper does not state;
    pinned by brute force over read/write orders in the tests)."""
    return 3 * rate if has_delay else 2 * rate


def write_slots(k: int, r: int):
    s = 1 + (k * r) % (3 * r)
    return list(range(s, s + r))


def read_slots(k: int, r: int):
    s = (k * r) % (3 * r)
    return list(range(s, s + r))


class DoubleBuffer:
    """Sequential model of the buffer of a channel without a delay token (Eq. 1,
    first case): 2r slots, write and read k both use slots (k r mod 2r) ... + r - 1."""

    def __init__(self, r: int):
        self.r = r
        self.slots = [None] * (2 * r)
        self.nw = 0
        self.nr = 0

    def write(self, tokens):
        assert len(tokens) == self.r
        s = (self.nw * self.r) % (2 * self.r)
        self.slots[s:s + self.r] = list(tokens)
        self.nw += 1

    def read(self):
        s = (self.nr * self.r) % (2 * self.r)
        self.nr += 1
        return self.slots[s:s + self.r]

    def unread(self) -> int:
        return self.nw * self.r - self.nr * self.r


class TripleBuffer:
    """Sequential model of the Fig. 2 buffer: alternating whole-window writes and reads."""

    def __init__(self, r: int, delay_token):
        self.r = r
        self.slots = [None] * (3 * r + 1)
        self.slots[0] = delay_token
        self.nw = 0
        self.nr = 0

    def write(self, tokens):
        assert len(tokens) == self.r
        ws = write_slots(self.nw, self.r)
        for s, t in zip(ws, tokens):
            self.slots[s] = t
        if ws[-1] == 3 * self.r:
            self.slots[0] = self.slots[3 * self.r]
        self.nw += 1

    def read(self):
        out = [self.slots[s] for s in read_slots(self.nr, self.r)]
        self.nr += 1
        return out

    def unread(self) -> int:
        """Tokens written (the delay token included) and not yet read."""
        return 1 + self.nw * self.r - self.nr * self.r
