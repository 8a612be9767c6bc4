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


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every parameter struct of the header has the same size and field offsets
    under gcc (plain C99) as in the ctypes binding."""
    import shutil
    import subprocess
    import pytest
    from paper_1611_03226_b300 import _lib as L
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"df_dpd_params": L.DpdParams, "df_md_params": L.MdParams, "df_img_params": L.ImgParams,
               "df_channel_info_t": L.ChannelInfo, "df_feed": L.Feed, "df_drain": L.Drain}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "dfgpu.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_every_declared_function_cites_its_passage():
    """Each entry point's comment names the passage of the paper that defines
    the operation (a section, equation, figure or table), or says that the paper
    has no counterpart."""
    cite = re.compile(r"(Sec\.\s*\d|Eq\.\s*\d|Fig\.\s*\d|Table\s*\d|no counterpart)")
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        # block comments: those that open a line (not a field's trailing comment)
        comments = [(m.start(), m.end(), m.group(0)) for m in re.finditer(r"/\*.*?\*/", text, flags=re.S)
                    if text[text.rfind("\n", 0, m.start()) + 1:m.start()].strip() == ""]
        code = re.sub(r"/\*.*?\*/", lambda m: " " * len(m.group(0)), text, flags=re.S)
        for m in re.finditer(r"\b(df_[a-z0-9_]+)\s*\(", code):
            before = [c for c in comments if c[1] <= m.start()]
            assert before, m.group(1)
            last = before[-1][2]
            assert cite.search(last), f"{m.group(1)}: no citation in its comment"
