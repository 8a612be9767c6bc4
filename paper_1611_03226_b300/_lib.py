"""ctypes binding of libdfgpu.so (argument marshalling only).

The library must have been built (``python -m paper_1611_03226_b300.build`` or
``__graft_entry__.build()``); importing this module without it raises, so no
caller can silently fall back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdfgpu.so")

DF_OK, DF_EINVAL, DF_ENOMEM, DF_EFULL, DF_EEMPTY, DF_ESTATE = 0, -1, -2, -3, -4, -5
DF_EDEADLOCK, DF_ETIMEOUT, DF_ECUDA, DF_ENOTSUP = -6, -7, -8, -9
DF_SOURCE, DF_SINK, DF_COPY, DF_DPD, DF_DPD_POLY, DF_DPD_FIR, DF_DPD_ADD, DF_MD = range(1, 9)
DF_GAUSS5, DF_THRES, DF_MED5 = 9, 10, 11
DF_RUN_ASYNC, DF_RUN_GRAPH, DF_RUN_PERSISTENT, DF_RUN_NO_BATCH = 1, 2, 4, 8
DF_IO_CONCURRENT = 1
DF_CAPACITY_EQ1 = 0
DF_LAYOUT_RING, DF_LAYOUT_EQ1 = 0, 1
DF_MAX_BRANCHES, DF_MAX_TAPS = 16, 32
DF_PROF_STEP, DF_PROF_DPD_BODY, DF_PROF_MD_MAIN, DF_PROF_COPY_BODY = 0, 1, 2, 3


class DpdParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("M", C.c_int32), ("orders", C.c_int32 * DF_MAX_BRANCHES),
                ("block_len", C.c_uint32), ("branch", C.c_int32), ("h", C.POINTER(C.c_float))]


class MdParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("threshold", C.c_int32),
                ("tile", C.c_int32)]


class ImgParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("threshold", C.c_int32)]


class ChannelInfo(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("slots", C.c_uint64), ("buffer_bytes", C.c_uint64),
                ("token_bytes", C.c_uint32), ("rate", C.c_uint32), ("initial_tokens", C.c_uint32),
                ("layout", C.c_int32)]


class Feed(C.Structure):
    _fields_ = [("source", C.c_int32), ("data", C.c_void_p), ("n_tokens", C.c_uint64),
                ("batch", C.c_uint64)]


class Drain(C.Structure):
    _fields_ = [("sink", C.c_int32), ("data", C.c_void_p), ("max_tokens", C.c_uint64),
                ("batch", C.c_uint64), ("n_popped", C.c_uint64)]


class DfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        detail = f" [{lib.df_last_error().decode()}]" if status == DF_ECUDA else ""
        super().__init__(f"{what}: {status_str(status)} ({status}){detail}")


_P = C.c_void_p
_PROTOS = {
    "df_net_create": (C.c_int32, [C.POINTER(_P), C.c_int, _P]),
    "df_net_destroy": (None, [_P]),
    "df_actor_add": (C.c_int32, [_P, C.c_int32, _P, C.c_size_t, C.POINTER(C.c_int32)]),
    "df_channel_connect": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint32,
                                       C.c_uint32, C.c_uint32, C.c_uint32, _P,
                                       C.POINTER(C.c_int32)]),
    "df_net_finalize": (C.c_int32, [_P]),
    "df_push": (C.c_int32, [_P, C.c_int32, _P, C.c_uint64, C.POINTER(C.c_uint64)]),
    "df_run": (C.c_int32, [_P, C.c_int64, C.POINTER(C.c_uint64)]),
    "df_run_ex": (C.c_int32, [_P, C.c_int64, C.c_uint32, C.POINTER(C.c_uint64)]),
    "df_sync": (C.c_int32, [_P, C.POINTER(C.c_uint64)]),
    "df_pop": (C.c_int32, [_P, C.c_int32, _P, C.c_uint64, C.POINTER(C.c_uint64)]),
    "df_push_ex": (C.c_int32, [_P, C.c_int32, _P, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64)]),
    "df_pop_ex": (C.c_int32, [_P, C.c_int32, _P, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64)]),
    "df_channel_info": (C.c_int32, [_P, C.c_int32, C.POINTER(ChannelInfo)]),
    "df_stream": (C.c_int32, [_P, C.POINTER(Feed), C.c_int32, C.POINTER(Drain), C.c_int32, C.c_uint32,
                              C.c_int64, C.POINTER(C.c_uint64)]),
    "df_channel_peek_slots": (C.c_int32, [_P, C.c_int32, C.c_uint64, C.c_uint64, C.c_void_p]),
    "df_channel_counters": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_uint64),
                                        C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "df_dpd_set_tile": (C.c_int32, [_P, C.c_int32, C.c_uint32, C.c_uint32]),
    "df_autotune": (C.c_int32, [_P, C.POINTER(C.c_uint64)]),
    "df_dpd_get_tile": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "df_status_str": (C.c_char_p, [C.c_int32]),
    "df_set_wait_limit": (C.c_int32, [_P, C.c_int64]),
    "df_selftest_wait_timeout": (C.c_int32, [_P, C.c_int64]),
    "df_last_error": (C.c_char_p, []),
    "df_profile_enable": (C.c_int32, [_P, C.c_int32]),
    "df_profile_get": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "df_dpd_forward": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                   C.POINTER(C.c_int32), _P, _P]),
    "df_dpd_backward": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int32), _P, _P, _P, _P]),
    "df_dpd_backward_scratch_elems": (C.c_uint64, [C.c_uint64, C.c_int32, C.c_int32]),
    "df_dpd_forward_f64": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                       C.POINTER(C.c_int32), _P, _P]),
    "df_dpd_backward_f64": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                        C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
    "df_dpd_backward_scratch": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                            C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
    "df_dpd_mse_partial_elems": (C.c_uint64, [C.c_uint64]),
    "df_dpd_mse_forward": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                       C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
    "df_dpd_mse_forward_f64": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                           C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
    "df_dpd_mse_backward": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                        C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
    "df_dpd_mse_backward_f64": (C.c_int32, [_P, C.c_uint64, _P, C.c_int32, C.c_int32,
                                            C.POINTER(C.c_int32), _P, _P, _P, _P, C.c_uint64, _P]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1611_03226_b300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


def status_str(s: int) -> str:
    return lib.df_status_str(s).decode()


def check(status: int, what: str):
    if status != DF_OK:
        raise DfError(status, what)
