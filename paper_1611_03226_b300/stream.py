"""Host actors in threads of their own beside the GPU actors (the paper's
heterogeneous execution, Sec. 3.3 and 4): producer threads push token batches
into the sources and consumer threads pop the sinks while the calling thread
runs engine steps.  Pushes and pops use the network's I/O streams
(DF_IO_CONCURRENT), so their copies overlap the step kernels and each other.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import _lib as L


def stream(net, feeds, sinks, flags=0, poll_s=50e-6):
    """Run `net` to completion while host threads feed and drain it.

    feeds: {source actor: iterable of token batches (host or device buffers)};
    every batch is pushed whole, retried while the channels lack space.
    sinks: {sink actor: tokens per pop} keeps every popped batch (returned as
    numpy byte arrays), or {sink actor: (tokens per pop, buffer)} pops into one
    reused buffer (pinned host memory for full-speed copies) and keeps only the
    number of tokens.  Returns ({sink: list of arrays or token count}, steps).
    """
    errors = []
    producers_done = threading.Event()
    stop_consumers = threading.Event()
    out = {s: ([] if isinstance(v, int) else 0) for s, v in sinks.items()}

    def produce(src, batches):
        try:
            for b in batches:
                while True:
                    try:
                        net.push(src, b, concurrent=True)
                        break
                    except L.DfError as e:
                        if e.status != L.DF_EFULL:
                            raise
                        time.sleep(poll_s)
        except BaseException as e:  # reported to the caller
            errors.append(e)

    def consume(sink, spec):
        try:
            while True:
                if isinstance(spec, int):
                    got = net.pop(sink, max_tokens=spec, concurrent=True)
                    n = len(got)
                    if n:
                        out[sink].append(got.copy())
                else:
                    per_pop, buf = spec
                    got = net.pop(sink, max_tokens=per_pop, out=buf, concurrent=True)
                    n = got[1] if isinstance(got, tuple) else len(got)
                    out[sink] += n if isinstance(got, tuple) else n // net.chan_tok[net.actor_in[sink][0]]
                if n:
                    continue
                if stop_consumers.is_set():
                    return
                time.sleep(poll_s)
        except BaseException as e:
            errors.append(e)

    ptv = [threading.Thread(target=produce, args=(s, b)) for s, b in feeds.items()]
    ctv = [threading.Thread(target=consume, args=(s, n)) for s, n in sinks.items()]
    for t in ptv + ctv:
        t.start()
    steps = 0
    try:
        while not errors:
            fired = net.run(1, flags)
            steps += 1
            if fired or any(t.is_alive() for t in ptv):
                if not fired:
                    time.sleep(poll_s)
                continue
            # sources done and a step fired nothing.  A full sink may have held an
            # actor back: once every sink is drained, one more step decides.
            if all(net.counters(net.actor_in[s][0])[2] == 0 for s in sinks):
                steps += 1
                if net.run(1, flags) == 0:
                    break
            else:
                time.sleep(poll_s)
    finally:
        for t in ptv:
            t.join()
        stop_consumers.set()
        for t in ctv:
            t.join()
    if errors:
        raise errors[0]
    return out, steps
