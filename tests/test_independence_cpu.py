"""The oracle and the CUDA path are independent, and the product path has no
fallback.

The oracle is test infrastructure: the package never imports it, and the two
share no source, header or table.  Only the seeded input generators
(``synth.py``, no reduction arithmetic) serve both.  Without its CUDA library
the package raises instead of computing anything another way.
"""
import importlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2008_11486_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "_build" in d or "_lib" in d or "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _code(path):
    with open(path) as f:
        src = f.read()
    # comments and docstrings may name the other side; only code counts
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = re.sub(r'"""(.*?)"""', " ", src, flags=re.S)
    return re.sub(r"#[^\n]*", " ", src) if path.endswith(".py") else src


def test_package_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        assert not re.search(r"^\s*(import|from)\s+oracle\b", _code(path), flags=re.M), path


def test_cuda_sources_and_oracle_share_nothing():
    for path in _files(PKG, (".cu", ".cuh", ".h")):
        code = _code(path)
        assert "oracle" not in code, path
    for path in _files(ORACLE, (".c", ".h", ".py")):
        code = _code(path)
        assert "paper_2008_11486_gb300" not in code and "irp.h" not in code, path
        assert not re.search(r"\birp_[a-z]", code), path  # no library call
        assert not re.search(r'#include\s+"(?!oracle\.h")', code), path


def test_only_the_input_generators_are_shared():
    # the generators hold no step of the reduction: no calibration formula,
    # no resampling, no clipping
    code = _code(os.path.join(PKG, "synth.py"))
    assert "import oracle" not in code and "_binding" not in code and "core" not in code
    for word in ("kappa", "bspline", "flat_norm", "median(", "sort("):
        assert word not in code, word


def test_the_package_raises_without_its_cuda_library(monkeypatch, tmp_path):
    from paper_2008_11486_gb300 import _binding as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing" / "libirp.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()
    core = importlib.import_module("paper_2008_11486_gb300.core")
    with pytest.raises(RuntimeError):
        core.profile_enable(True)
