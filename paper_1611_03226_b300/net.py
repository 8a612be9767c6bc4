"""Python face of the C ABI: build a network, push, run, pop (marshalling only).

Host buffers are numpy arrays; device buffers are torch CUDA tensors.  Every
call goes straight to libdfgpu.so; nothing here computes on the data.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _ptr(buf):
    """(address, nbytes) of a C-contiguous numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data, buf.nbytes
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), buf.numel() * buf.element_size()
    raise TypeError(f"unsupported buffer {type(buf)}")


class Net:
    """One network.  ``stream`` is a cudaStream_t handle (int) the network runs
    on; None or 0 lets the network create its own stream (the legacy default
    stream is never used)."""

    def __init__(self, device: int = 0, stream=None):
        h = C.c_void_p()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        s = C.c_void_p(stream) if stream else None
        L.check(L.lib.df_net_create(C.byref(h), device, s), "df_net_create")
        self.h = h
        self.chan_tok = {}
        self.actor_out = {}      # actor -> {port: ch}
        self.actor_in = {}

    def close(self):
        if self.h:
            L.lib.df_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- construction ----
    def _add(self, kind, params=None):
        aid = C.c_int32()
        if params is None:
            L.check(L.lib.df_actor_add(self.h, kind, None, 0, C.byref(aid)), "df_actor_add")
        else:
            L.check(L.lib.df_actor_add(self.h, kind, C.byref(params), C.sizeof(params),
                                       C.byref(aid)), "df_actor_add")
        return aid.value

    def add_source(self):
        return self._add(L.DF_SOURCE)

    def add_sink(self):
        return self._add(L.DF_SINK)

    def add_copy(self):
        return self._add(L.DF_COPY)

    def add_dpd(self, h, orders, block_len, kind=L.DF_DPD, branch=0):
        h = np.ascontiguousarray(h, np.complex64)
        K, M = h.shape
        p = L.DpdParams()
        p.K, p.M, p.block_len, p.branch = K, M, block_len, branch
        for k, o in enumerate(orders):
            p.orders[k] = int(o)
        hf = h.view(np.float32).reshape(-1)
        p.h = hf.ctypes.data_as(C.POINTER(C.c_float))
        aid = self._add(kind, p)
        del hf
        return aid

    def add_md(self, width, height, threshold=25, tile=16):
        p = L.MdParams(width, height, threshold, tile)
        return self._add(L.DF_MD, p)

    # the paper's motion pipeline (Sec. 4.1): Gauss -> Thres -> Med on u8 frames
    def add_gauss5(self, width, height):
        return self._add(L.DF_GAUSS5, L.ImgParams(width, height, 0))

    def add_thres(self, width, height, threshold=20):
        return self._add(L.DF_THRES, L.ImgParams(width, height, threshold))

    def add_med5(self, width, height):
        return self._add(L.DF_MED5, L.ImgParams(width, height, 0))

    def connect(self, src, src_port, dst, dst_port, token_bytes, rate, capacity, initial=0,
                initial_data=None):
        """capacity="eq1" (DF_CAPACITY_EQ1) gives the paper's layout: Eq. 1 sizes the
        buffer and a delay channel follows the access pattern of Fig. 2."""
        if capacity == "eq1":
            capacity = L.DF_CAPACITY_EQ1
        ch = C.c_int32()
        ptr = None
        if initial_data is not None:
            initial_data = np.ascontiguousarray(initial_data)
            if initial_data.nbytes != initial * token_bytes:
                raise ValueError("initial_data size mismatch")
            ptr = C.c_void_p(initial_data.ctypes.data)
        L.check(L.lib.df_channel_connect(self.h, src, src_port, dst, dst_port, token_bytes, rate,
                                         capacity, initial, ptr, C.byref(ch)),
                "df_channel_connect")
        self.chan_tok[ch.value] = token_bytes
        self.actor_out.setdefault(src, {})[src_port] = ch.value
        self.actor_in.setdefault(dst, {})[dst_port] = ch.value
        return ch.value

    def finalize(self):
        L.check(L.lib.df_net_finalize(self.h), "df_net_finalize")

    # ---- execution ----
    def push(self, src, buf, n_tokens=None, concurrent=False):
        """Copy whole tokens into every output channel of source `src` (all or
        nothing).  concurrent=True runs the copy on the network's push stream, so
        it may overlap a run() in another thread (df_push_ex, DF_IO_CONCURRENT)."""
        addr, nbytes = _ptr(buf)
        tok = self.chan_tok[self.actor_out[src][0]]
        if n_tokens is None:
            if nbytes % tok:
                raise ValueError("buffer is not a whole number of tokens")
            n_tokens = nbytes // tok
        elif n_tokens * tok > nbytes:
            raise ValueError("buffer too small")
        n = C.c_uint64()
        L.check(L.lib.df_push_ex(self.h, src, C.c_void_p(addr), n_tokens,
                                 L.DF_IO_CONCURRENT if concurrent else 0, C.byref(n)), "df_push")
        return n.value

    def run(self, n_steps=-1, flags=0):
        n = C.c_uint64()
        L.check(L.lib.df_run_ex(self.h, n_steps, flags, C.byref(n)), "df_run")
        return n.value

    def run_async(self, n_steps, flags=0):
        L.check(L.lib.df_run_ex(self.h, n_steps, flags | L.DF_RUN_ASYNC, None), "df_run")

    def sync(self):
        n = C.c_uint64()
        L.check(L.lib.df_sync(self.h, C.byref(n)), "df_sync")
        return n.value

    def pop(self, sink, max_tokens=None, out=None, dtype=np.uint8, concurrent=False):
        """Copy up to max_tokens tokens out of sink `sink`.  concurrent=True runs
        the copy on the network's pop stream (df_pop_ex, DF_IO_CONCURRENT); then
        `out` or `max_tokens` must be given."""
        ch = self.actor_in[sink][0]
        tok = self.chan_tok[ch]
        if out is None:
            if concurrent:
                if max_tokens is None:
                    raise ValueError("a concurrent pop needs out or max_tokens")
                n_max = max_tokens
            else:
                produced, consumed, occ = self.counters(ch)
                n_max = occ if max_tokens is None else min(max_tokens, occ)
            out = np.empty(n_max * tok, np.uint8)
        addr, nbytes = _ptr(out)
        cap = nbytes // tok
        n = C.c_uint64()
        L.check(L.lib.df_pop_ex(self.h, sink, C.c_void_p(addr),
                                cap if max_tokens is None else min(cap, max_tokens),
                                L.DF_IO_CONCURRENT if concurrent else 0, C.byref(n)),
                "df_pop")
        if isinstance(out, np.ndarray):
            return out[: n.value * tok].view(dtype)
        return out, n.value

    def stream(self, feeds, drains, flags=0, idle_limit_s=0.0):
        """Run to completion with the paper's host actors as native threads
        (df_stream): feeds {source: (buffer of tokens, tokens per push)}, drains
        {sink: (output buffer, tokens per pop)}.  Returns ({sink: tokens popped},
        steps run)."""
        fs = (L.Feed * max(1, len(feeds)))()
        keep = []
        for i, (src, (buf, batch)) in enumerate(feeds.items()):
            addr, nbytes = _ptr(buf)
            tok = self.chan_tok[self.actor_out[src][0]]
            if nbytes % tok:
                raise ValueError("feed is not a whole number of tokens")
            fs[i] = L.Feed(src, addr, nbytes // tok, batch)
            keep.append(buf)
        ds = (L.Drain * max(1, len(drains)))()
        for i, (snk, (buf, batch)) in enumerate(drains.items()):
            addr, nbytes = _ptr(buf)
            tok = self.chan_tok[self.actor_in[snk][0]]
            ds[i] = L.Drain(snk, addr, nbytes // tok, batch, 0)
            keep.append(buf)
        steps = C.c_uint64()
        L.check(L.lib.df_stream(self.h, fs, len(feeds), ds, len(drains), flags, int(idle_limit_s * 1e9),
                                C.byref(steps)), "df_stream")
        return {snk: ds[i].n_popped for i, snk in enumerate(drains)}, steps.value

    def channel_info(self, ch):
        """Layout and size of a channel: dict of capacity (most unread tokens), slots,
        buffer_bytes, token_bytes, rate, initial_tokens and layout ("ring" or "eq1")."""
        i = L.ChannelInfo()
        L.check(L.lib.df_channel_info(self.h, ch, C.byref(i)), "df_channel_info")
        d = {k: getattr(i, k) for k, _ in L.ChannelInfo._fields_}
        d["layout"] = "eq1" if i.layout == L.DF_LAYOUT_EQ1 else "ring"
        return d

    def peek_slots(self, ch, first=0, n=None):
        """Raw buffer slots of a channel (uint8 array of n slots x token bytes)."""
        info = self.channel_info(ch)
        if n is None:
            n = info["slots"] - first
        out = np.empty(n * info["token_bytes"], np.uint8)
        L.check(L.lib.df_channel_peek_slots(self.h, ch, first, n, C.c_void_p(out.ctypes.data)),
                "df_channel_peek_slots")
        return out.reshape(n, info["token_bytes"])

    def counters(self, ch):
        p, c, o = C.c_uint64(), C.c_uint64(), C.c_uint64()
        L.check(L.lib.df_channel_counters(self.h, ch, C.byref(p), C.byref(c), C.byref(o)),
                "df_channel_counters")
        return p.value, c.value, o.value

    def set_wait_limit(self, ns):
        L.check(L.lib.df_set_wait_limit(self.h, int(ns)), "df_set_wait_limit")

    def selftest_wait_timeout(self, ns):
        """Status left by a grid barrier that can only end by its time limit."""
        return L.lib.df_selftest_wait_timeout(self.h, int(ns))

    def profile(self, on=True):
        L.check(L.lib.df_profile_enable(self.h, 1 if on else 0), "df_profile_enable")

    def profile_get(self, what):
        ms, n = C.c_double(), C.c_uint64()
        L.check(L.lib.df_profile_get(self.h, what, C.byref(ms), C.byref(n)), "df_profile_get")
        return ms.value, n.value

    def autotune(self):
        n = C.c_uint64()
        L.check(L.lib.df_autotune(self.h, C.byref(n)), "df_autotune")
        return n.value

    def get_tile(self, actor):
        t, th = C.c_uint32(), C.c_uint32()
        L.check(L.lib.df_dpd_get_tile(self.h, actor, C.byref(t), C.byref(th)), "df_dpd_get_tile")
        return t.value, th.value

    def set_tile(self, actor, tile, threads):
        L.check(L.lib.df_dpd_set_tile(self.h, actor, tile, threads), "df_dpd_set_tile")
