"""The oracle and the library stay independent: nothing in the package or
the input generators imports the oracle or names a file under it, and the
oracle imports neither the package nor torch and loads no compiled code."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(sub, exts):
    for d, _, fs in os.walk(os.path.join(ROOT, sub)):
        if "__pycache__" in d or "_lib" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_and_inputs_do_not_import_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|oracle/", re.M)
    bad = [p for sub in ("paper_2504_21440_gb300", "workloads")
           for p in _files(sub, (".py", ".cu", ".cuh", ".cpp", ".h"))
           if pat.search(open(p, encoding="utf-8").read())]
    assert bad == []


def test_oracle_uses_neither_the_library_nor_compiled_code():
    pat = re.compile(r"^\s*(from|import)\s+(paper_2504_21440_gb300|ctypes|torch|cffi|numba|cupy)\b"
                     r"|libqtl|CDLL|\.so\b", re.M)
    bad = [p for p in _files("oracle", (".py",)) if pat.search(open(p, encoding="utf-8").read())]
    assert bad == []
