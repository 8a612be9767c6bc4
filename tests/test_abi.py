"""The C-ABI library loads and exports every entry point include/dfgpu.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(df_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1611_03226_b300 import _lib
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(_lib.lib, n)]
    assert not missing, missing


def test_status_strings_and_no_gpu_behaviour():
    import torch
    from paper_1611_03226_b300 import _lib as L
    assert L.status_str(L.DF_EFULL) == "channel full"
    assert L.status_str(12345) == "unknown status"
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert L.lib.df_net_create(ctypes.byref(h), 0, None) == L.DF_EINVAL
    L.lib.df_net_destroy(None)        # NULL-safe


def test_param_struct_layout_matches_header():
    from paper_1611_03226_b300 import _lib as L
    # int32 K, M, orders[16], uint32 block_len, int32 branch, then an 8-byte aligned pointer
    assert ctypes.sizeof(L.DpdParams) == 4 * (2 + 16 + 2) + 8
    assert ctypes.sizeof(L.MdParams) == 16
