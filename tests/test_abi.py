"""The C ABI library builds for sm_103a and exports every symbol af.h declares.

CPU only: the library is compiled (nvcc cross-compiles without a GPU) and
loaded, but no compute call is made.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(af_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_declared_symbols():
    from paper_2506_04857_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "af_step" in syms and "af_create" in syms and len(syms) >= 15
    for name in syms:
        assert hasattr(lib, name), name


def test_binding_has_the_same_names():
    import paper_2506_04857_gb300 as af
    for name in declared_symbols():
        assert callable(getattr(af, name)), name


def test_no_cpu_fallback_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2506_04857_gb300 as af
    with pytest.raises(af.AFError):
        af.af_create(8, 8, 1.4, af.AF_BC_PERIODIC)
