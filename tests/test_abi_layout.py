"""The Python binding's ctypes structures mirror the C structures of
include/mrhs.h: a small C program compiled here with the host compiler prints
sizeof and offsetof of every field, and each must equal the ctypes layout.
(A mismatch would make the binding pass garbage parameters to the library.)"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2211_13719_gb300 import mrhs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "mrhs_mg_params": mrhs.MgParams,
    "mrhs_solve_stats": mrhs.SolveStats,
    "mrhs_server_params": mrhs.ServerParams,
    "mrhs_request_stats": mrhs.RequestStats,
    "mrhs_tune_entry": mrhs.TuneEntry,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mrhs.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        s, f, v = line.split()
        layout[(s, f)] = int(v)
    return layout


def test_ctypes_structures_match_the_c_header(tmp_path):
    layout = _c_layout(tmp_path)
    for cname, cls in STRUCTS.items():
        assert ctypes.sizeof(cls) == layout[(cname, "sizeof")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == layout[(cname, fname)], f"{cname}.{fname}"
