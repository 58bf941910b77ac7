"""The Python binding's ctypes structures have the layout of include/mb.h:
a small C program compiled against the header prints every size and field
offset, and each must match the binding's.  Host only (no GPU, no CUDA)."""
import os
import shutil
import subprocess
import tempfile

import ctypes
import pytest

from paper_2007_00745_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "mb_window": _lib.mb_window,
    "mb_item": None,
    "mb_cta_trace": None,
    "mb_opts": _lib.mb_opts,
    "mb_view": _lib.mb_view,
    "mb_request": _lib.mb_request,
    "mb_req_stats": _lib.mb_req_stats,
    "mb_serve_counters": _lib.mb_serve_counters,
    "mb_run_stats": _lib.mb_run_stats,
}


def _c_layout():
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mb.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        if cls is not None:
            for f, _ in cls._fields_:
                lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ['  printf("mb_item tile %zu\\n", offsetof(mb_item, tile));',
              '  printf("mb_item row0 %zu\\n", offsetof(mb_item, row0));',
              '  printf("mb_item rows %zu\\n", offsetof(mb_item, rows));',
              '  printf("mb_cta_trace items %zu\\n", offsetof(mb_cta_trace, items));',
              "  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        s, f, v = line.split()
        res[(s, f)] = int(v)
    return res


def test_ctypes_structures_match_the_header():
    c = _c_layout()
    for name, cls in STRUCTS.items():
        if cls is None:
            continue
        assert ctypes.sizeof(cls) == c[(name, "sizeof")], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(name, f)], (name, f)


def test_fixed_size_records():
    c = _c_layout()
    assert c[("mb_item", "sizeof")] == 8 and c[("mb_item", "rows")] == 6
    assert c[("mb_cta_trace", "sizeof")] == 24 and c[("mb_cta_trace", "items")] == 20
