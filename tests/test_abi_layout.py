"""The ctypes structures of the Python binding have the layout of the C
structures in include/lpk.h (sizes and field offsets, measured by compiling a
small C program against the header with the host compiler).  CPU only."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1604_07491_gb300 import lpk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "lpk_matrix": lpk.Matrix,
    "lpk_options": lpk.Options,
    "lpk_info": lpk.Info,
    "lpk_krylov_info": lpk.KrylovInfo,
    "lpk_stats": lpk.Stats,
    "lpk_server_config": lpk.ServerConfig,
    "lpk_request_result": lpk.RequestResult,
    "lpk_server_stats_t": lpk.ServerStats,
}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lpk.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    got = {}
    for line in out.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    return got


def test_ctypes_structures_match_the_header(tmp_path):
    c = c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert c[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert c[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
