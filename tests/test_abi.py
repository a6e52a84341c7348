"""The C-ABI library builds for sm_103a, loads, and exports every call that
include/*.h declares (no GPU needed: nothing is computed)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    n = declared()
    for core in ("fr_create", "fr_set_mesh", "fr_set_lights", "fr_forward", "fr_backward", "fr_loss",
                 "fr_render", "fr_sync_status", "fr_last_error", "fr_destroy"):
        assert core in n


def test_library_exports_every_declared_symbol():
    from paper_2101_05356_gb300 import build
    lib = build.build()
    L = ctypes.CDLL(lib)
    missing = [n for n in sorted(declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2101_05356_gb300 import facert
    monkeypatch.setattr(facert, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(facert, "_lib", None)
    import pytest
    with pytest.raises(RuntimeError):
        facert.lib()


def test_oracle_is_not_imported_by_the_product_path():
    pkg = os.path.join(ROOT, "paper_2101_05356_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        txt = open(f, errors="ignore").read()
        assert "import oracle" not in txt and "from oracle" not in txt and "oracle.h" not in txt, f
