"""CPU check of the grid multigrid's index arithmetic: a host program built against
csrc/xpbd_mg_index.h (the functions the kernels call) checks that the diagonal lines and
the point colours cover every vertex once, that same-colour lines or points never interact
through the 5 x 5 stencil, that the compact line-residual items cover each colour once,
that the prolongation weights are a partition of unity inside the index ranges the
restriction and prolongation kernels visit, and that the carved workspace ends exactly at
its allocation with a coarsest level of at most 16 vertices."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_multigrid_index_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "mg_index_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2301_01396_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "mg_index_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
