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


def test_every_entry_point_rejects_null_arguments(L):
    """Each call checks its pointers and scalars before it touches the device."""
    lib = L.lib()
    h = (ctypes.c_double * 3)(0, 0, 0)
    fake = ctypes.c_void_p(16)
    opts = L.make_opts()
    E = (ctypes.c_double * 5)()
    mavg = (ctypes.c_double * 3)()
    ARG = L.MM_ERR_ARG
    assert lib.mm_energy(None, fake, h, E, None) == ARG
    assert lib.mm_hysteresis_sweep(None, fake, h, 1, 0, ctypes.byref(opts), mavg, None, None) == ARG
    assert lib.mm_energy_gradient(None, fake, h, 1.0, fake, None) == ARG
    assert lib.mm_hessian_vec(None, fake, h, fake, fake, None) == ARG
    assert lib.mm_adjoint_dK(None, fake, h, fake, fake, 1e-8, 100, None, None, None) == ARG
    assert lib.mm_set_anisotropy(None, fake, None) == ARG
    assert lib.mm_hysteresis_sweep_mixed(None, None, fake, h, 1, 0, ctypes.byref(opts), ctypes.byref(opts),
                                         mavg, None, None, None) == ARG
    out = ctypes.c_void_p()
    assert lib.mm_batch_create(None, 1, ctypes.byref(out)) == ARG
    assert out.value is None
    assert lib.mm_batch_destroy(None) == L.MM_OK
    assert lib.mm_batch_sweep(None, None, h, 1, 0, ctypes.byref(opts), mavg, None, None) == ARG
    info = L.mm_info()
    assert lib.mm_problem_info(None, ctypes.byref(info)) == ARG
    ms = (ctypes.c_double * 8)()
    names = (ctypes.c_char_p * 8)()
    cnt = ctypes.c_int()
    assert lib.mm_kernel_times(None, fake, h, 1, ms, names, ctypes.byref(cnt), None) == ARG
    g = L.make_grid(4, 4, 1, 1e-9, 1e-9, 1e-9)
    assert lib.mm_newell_static(ctypes.byref(g), None, None) == ARG
    assert lib.mm_newell_static(None, fake, None) == ARG


def test_newell_static_refuses_grids_past_its_buffer(L):
    lib = L.lib()
    big = L.make_grid(4096, 4096, 64, 1e-9, 1e-9, 1e-9)
    assert lib.mm_newell_static(ctypes.byref(big), ctypes.c_void_p(16), None) == L.MM_ERR_UNSUPPORTED
    # nx + 1 would overflow a 32-bit int: the lattice count is taken in 64 bits
    huge = L.make_grid(2**31 - 1, 1, 1, 1e-9, 1e-9, 1e-9)
    assert lib.mm_newell_static(ctypes.byref(huge), ctypes.c_void_p(16), None) in (L.MM_ERR_UNSUPPORTED,
                                                                                  L.MM_ERR_ARG)
    assert isinstance(L.mm_status_string(L.MM_ERR_UNSUPPORTED), str)


def test_binding_checks_host_outputs_before_the_call(L):
    """Shapes, dtypes and lengths the library cannot check are checked in the
    binding; a null problem handle then gets MM_ERR_ARG from the library."""
    import numpy as np
    prob = L.Problem(None, L.make_grid(4, 4, 1, 1e-9, 1e-9, 1e-9), L.MM_FP64)
    m = np.zeros(prob.shape)
    H = np.zeros((5, 3))
    for bad in (np.zeros((4, 3)), np.zeros((5, 3), np.float32), np.zeros((3, 5)).T, np.zeros(15)):
        with pytest.raises(ValueError):
            L.mm_hysteresis_sweep(prob, m, H, mavg=bad)
        with pytest.raises(ValueError):
            L.mm_hysteresis_sweep_mixed(prob, prob, m, H, mavg=bad)
    ro = np.zeros((5, 3))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        L.mm_hysteresis_sweep(prob, m, H, mavg=ro)
    with pytest.raises(L.MMError) as e:
        L.mm_hysteresis_sweep(prob, m, H, mavg=np.zeros((5, 3)))
    assert e.value.status == L.MM_ERR_ARG
    with pytest.raises(TypeError):
        L.mm_hysteresis_sweep(prob, m.astype(np.float32), H)
    batch = L.Batch(None, [prob, prob])
    with pytest.raises(ValueError):
        L.mm_batch_sweep(batch, [m], H)
    with pytest.raises(L.MMError):
        L.mm_batch_sweep(batch, [m, m], H)


def test_batch_refuses_a_repeated_problem(L):
    # the repeat is found before any problem is looked at, so placeholder
    # handles suffice here
    lib = L.lib()
    out = ctypes.c_void_p()
    same = (ctypes.c_void_p * 3)(16, 32, 16)
    assert lib.mm_batch_create(same, 3, ctypes.byref(out)) == L.MM_ERR_ARG
    assert out.value is None
    assert lib.mm_batch_create(same, 0, ctypes.byref(out)) == L.MM_ERR_ARG
