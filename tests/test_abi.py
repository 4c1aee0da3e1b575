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
            names.update(re.findall(r"\b(af(?:1d)?_[a-z_0-9]+)\s*\(", text))
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


def test_grid_limits_are_rejected_before_any_device_call():
    """Grids beyond the launch shape (ny + 1 > 4 * 65535) or the adjoint's DoF
    ids ((nx + 1)(ny + 1) >= 2^28) are refused with AF_EINVAL, for a context and
    for a batch run, before CUDA is touched (this runs without a GPU)."""
    from paper_2506_04857_gb300 import build
    lib = ctypes.CDLL(build.build())
    out = ctypes.c_void_p()
    for nx, ny in ((4, 262140), (20000, 20000), (3, 16), (16, 3)):
        assert lib.af_create(nx, ny, ctypes.c_double(1.4), 1, ctypes.byref(out)) == -1, (nx, ny)
        assert not out.value
        NX, NY = (ctypes.c_int * 2)(16, nx), (ctypes.c_int * 2)(16, ny)
        G, BC = (ctypes.c_double * 2)(1.4, 1.4), (ctypes.c_int * 2)(1, 1)
        assert lib.af_batch_create(2, NX, NY, G, BC, ctypes.byref(out)) == -1, (nx, ny)
