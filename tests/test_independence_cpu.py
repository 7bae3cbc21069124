"""Structural rules between the product and its checker (CPU only).

* The oracle and the CUDA path share no code: nothing under ``oracle/``
  imports the package, and nothing in the package imports ``oracle``.  The
  only module both sides use is the seeded input generator ``synth.py``,
  which holds none of the transform's arithmetic.
* Only the tests, the smoke run and the benchmark's CPU legs reach the
  oracle.
* The product path has no CPU fallback: without the built library the
  binding raises instead of computing anything.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2006_08435_gb300")


def _py_imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_oracle_does_not_use_the_package():
    for f in _files(os.path.join(ROOT, "oracle"), (".py",)):
        assert "paper_2006_08435_gb300" not in _py_imports(f), f
    for f in _files(os.path.join(ROOT, "oracle"), (".c", ".h")):
        src = open(f, encoding="utf-8").read()
        assert not re.search(r'#include\s+"[^"]*(csrc|fft3d)', src), f


def test_package_does_not_use_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _py_imports(f), f
    for f in _files(PKG, (".cu", ".cuh", ".h")):
        src = open(f, encoding="utf-8").read()
        assert not re.search(r'#include\s+"[^"]*oracle', src), f


def test_generator_holds_no_transform_arithmetic():
    """synth.py draws numbers and lays out grids; it calls no FFT or DFT."""
    src = open(os.path.join(PKG, "synth.py"), encoding="utf-8").read()
    assert "fft" not in src.lower().replace("fft3d", "")
    assert "oracle" not in _py_imports(os.path.join(PKG, "synth.py"))


def test_only_checkers_reach_the_oracle():
    allowed = {os.path.join(ROOT, "bench.py"), os.path.join(ROOT, "__graft_entry__.py")}
    for f in _files(ROOT, (".py",)):
        rel = os.path.relpath(f, ROOT)
        if rel.startswith(("tests" + os.sep, "oracle" + os.sep, "_work" + os.sep, "baseline" + os.sep)):
            continue
        if "oracle" in _py_imports(f):
            assert f in allowed, rel


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2006_08435_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(Exception) as e:
        _lib.lib()
    assert "not built" in str(e.value) or "fallback" in str(e.value)
