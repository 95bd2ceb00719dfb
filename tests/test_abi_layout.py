"""The binding's ctypes structures have the C layout of include/diffxpbd.h: a small C
program compiled against the header prints sizeof and offsetof of every field the binding
declares, and both must agree (a field added to one side only, or in another order,
fails here on the CPU)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2301_01396_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "xpbd_model": binding.XpbdModel,
    "xpbd_params": binding.XpbdParams,
    "xpbd_grads": binding.XpbdGrads,
    "xpbd_implicit_opts": binding.XpbdImplicitOpts,
    "xpbd_kernel_stat": binding.XpbdKernelStat,
    "xpbd_request": binding.XpbdRequest,
    "xpbd_server_stats": binding.XpbdServerStats,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "diffxpbd.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    return got


def test_ctypes_structures_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, cls in STRUCTS.items():
        assert C.sizeof(cls) == c[(cname, "sizeof")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == c[(cname, fname)], (cname, fname)
