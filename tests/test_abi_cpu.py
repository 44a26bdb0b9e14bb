"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/qtl.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    from paper_2504_21440_gb300 import build
    lib_path = build.build()
    hdr = open(os.path.join(ROOT, "include", "qtl.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    hdr = re.sub(r"typedef[^;]*;", "", hdr)   # type names, e.g. the callback type
    names = sorted(set(re.findall(r"\b(qtl_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 12
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2504_21440_gb300 import qtl
    monkeypatch.setattr(qtl, "_lib", None)
    monkeypatch.setattr(qtl, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        qtl.load()
        raised = False
    except RuntimeError:
        raised = True
    assert raised


def test_host_side_strings_and_defaults():
    from paper_2504_21440_gb300 import qtl
    qtl.load()
    o = qtl.opts_default()
    assert o.method == 1 and o.precision == 0 and o.rtol == 1e-8 and o.atol == 1e-10
    assert qtl.strerror(qtl.QTL_ESTEP).startswith("step size")
    assert qtl.launch_count() == 0
