"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "diffxpbd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xpbd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("xpbd_create", "xpbd_forward", "xpbd_adjoint", "xpbd_destroy", "xpbd_loss"):
        assert f in names


def test_library_builds_and_exports_every_symbol():
    from paper_2301_01396_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2301_01396_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.lib()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2301_01396_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "xpbd_oracle" not in txt, f


def test_kernel_class_names_match_the_binding():
    """xpbd_kernel_class_name names every class the binding's profile table lists, in order."""
    from paper_2301_01396_gb300 import binding, build
    lib = ctypes.CDLL(build.build())
    lib.xpbd_kernel_class_name.restype = ctypes.c_char_p
    names = [lib.xpbd_kernel_class_name(i).decode() for i in range(len(binding.KERNEL_CLASSES))]
    assert tuple(names) == binding.KERNEL_CLASSES
    assert lib.xpbd_kernel_class_name(len(binding.KERNEL_CLASSES)) == b""
