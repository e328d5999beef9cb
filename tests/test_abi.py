"""The C-ABI library builds for sm_103a, loads, exports every entry point that
include/mm.h declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1405_2728_gb300 import build as mmbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    mmbuild.build()
    from paper_1405_2728_gb300 import mm
    return mm


def declared():
    txt = open(os.path.join(ROOT, "include", "mm.h")).read()
    return re.findall(r"MM_API\s+(?:const\s+)?\w+\s*\*?\s*(mm_\w+)\s*\(", txt)


def test_header_declares_the_boundary():
    names = set(declared())
    for n in ("mm_newell", "mm_setup_geometry", "mm_destroy", "mm_heff", "mm_energy", "mm_minimize",
              "mm_hysteresis_sweep", "mm_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.LIB_PATH)
    for n in declared():
        assert hasattr(lib, n), n


def test_status_strings(L):
    assert L.mm_status_string(0) == "ok"
    for s in range(-7, 0):
        assert L.mm_status_string(s) not in ("", "unknown status")
    assert L.mm_status_string(99) == "unknown status"


def test_host_side_argument_checks(L):
    lib = L.lib()
    out = ctypes.c_void_p()
    g = L.make_grid(4, 4, 1, 1e-9, 1e-9, 1e-9)
    mat = L.make_material(8e5, 1.3e-11, 500.0)
    assert lib.mm_setup_geometry(None, ctypes.byref(mat), 0, None, ctypes.byref(out)) == L.MM_ERR_ARG
    assert lib.mm_setup_geometry(ctypes.byref(g), None, 0, None, ctypes.byref(out)) == L.MM_ERR_ARG
    assert lib.mm_setup_geometry(ctypes.byref(g), ctypes.byref(mat), 7, None, ctypes.byref(out)) == L.MM_ERR_ARG
    bad = [L.make_grid(0, 4, 1, 1e-9, 1e-9, 1e-9), L.make_grid(4, 4, 1, -1e-9, 1e-9, 1e-9),
           L.make_grid(4, 4, 1, float("nan"), 1e-9, 1e-9)]
    for b in bad:
        assert lib.mm_setup_geometry(ctypes.byref(b), ctypes.byref(mat), 0, None, ctypes.byref(out)) == L.MM_ERR_ARG
        assert lib.mm_newell(ctypes.byref(b), ctypes.c_void_p(16), None) == L.MM_ERR_ARG
    for m in (L.make_material(0.0, 1e-11), L.make_material(8e5, -1.0), L.make_material(8e5, 1e-11, 1.0, (1, 1, 0))):
        assert lib.mm_setup_geometry(ctypes.byref(g), ctypes.byref(m), 0, None, ctypes.byref(out)) == L.MM_ERR_ARG
    assert out.value is None
    assert lib.mm_newell(ctypes.byref(g), None, None) == L.MM_ERR_ARG
    h = (ctypes.c_double * 3)(0, 0, 0)
    assert lib.mm_heff(None, ctypes.c_void_p(16), h, ctypes.c_void_p(16), None) == L.MM_ERR_ARG
    assert lib.mm_minimize(None, None, h, None, None, None) == L.MM_ERR_ARG
    assert lib.mm_destroy(None) == 0


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_1405_2728_gb300 import mm
    monkeypatch.setattr(mm, "_lib", None)
    monkeypatch.setattr(mm, "LIB_PATH", "/nonexistent/libmmgb.so")
    with pytest.raises(ImportError):
        mm.lib()
