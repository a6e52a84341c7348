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


# ctypes structures of the binding and the C structures they mirror
_STRUCTS = [("FrConfig", "fr_config"), ("FrMesh", "fr_mesh"), ("FrLightStage", "fr_light_stage"),
            ("FrAlbedoModel", "fr_albedo_model"), ("FrParams", "fr_params"), ("FrGrads", "fr_grads"),
            ("FrOptGroup", "fr_opt_group"), ("FrItem", "fr_item"), ("FrServerConfig", "fr_server_config"),
            ("FrRequest", "fr_request"), ("FrResult", "fr_result"), ("FrServerStats", "fr_server_stats")]


def test_header_compiles_as_c_and_cpp(tmp_path):
    import subprocess
    inc = os.path.join(ROOT, "include")
    for cc, std, lang in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")):
        src = tmp_path / ("t." + ("c" if lang == "c" else "cpp"))
        src.write_text('#include "facert.h"\nint main(void) { return 0; }\n')
        r = subprocess.run([cc, std, "-Wall", "-Werror", "-pedantic", "-fsyntax-only", "-I", inc, str(src)],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_structs_match_the_header(tmp_path):
    """Size and every field offset of the binding's ctypes structures equal
    the C compiler's for the header's structures (host ABI)."""
    import subprocess
    from paper_2101_05356_gb300 import facert
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "facert.h"', 'int main(void) {']
    for py, c in _STRUCTS:
        cls = getattr(facert, py)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (py, c))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (py, f[0], c, f[0]))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for py, _ in _STRUCTS:
        cls = getattr(facert, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for f in cls._fields_:
            assert got[(py, f[0])] == getattr(cls, f[0]).offset, (py, f[0])
