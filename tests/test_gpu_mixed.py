"""Mixed-precision sweep (extension): per field value an FP32 minimisation to
a loose tolerance, then FP64 from there to the final tolerance.  The loop
must match the plain FP64 loop the way two FP64 loops match each other
(switching field within one field step, remanence within 1e-3, the same
values up to the first switching event), and end every field value
converged to the final tolerance."""
import numpy as np
import pytest

from gpu_cases import dev
from paper_1405_2728_gb300 import inputs

pytestmark = pytest.mark.gpu


def loop_metrics(F, mavg):
    from oracle import micromag as om
    return om.loop_metrics(F, mavg)


def test_mixed_loop_matches_fp64_loop(mmlib):
    w = inputs.film_32x16x1()
    grid = mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    mat = mmlib.make_material(w.Ms, w.A, w.K)
    p64 = mmlib.mm_setup_geometry(grid, mat, mmlib.MM_FP64)
    p32 = mmlib.mm_setup_geometry(grid, mat, mmlib.MM_FP32)
    F = w.fields()
    m64 = dev(w.initial_m())
    st, mavg64, res64 = mmlib.mm_hysteresis_sweep(p64, m64, F, opts=mmlib.make_opts(tol=w.tol))
    assert st == mmlib.MM_OK
    mm_ = dev(w.initial_m())
    st, mavg, rl, rh = mmlib.mm_hysteresis_sweep_mixed(p32, p64, mm_, F, opts_lo=mmlib.make_opts(tol=1e-4, max_iter=20000),
                                                       opts_hi=mmlib.make_opts(tol=w.tol))
    assert st == mmlib.MM_OK and all(r.converged and r.max_torque < w.tol for r in rh)
    a, b = loop_metrics(F, mavg), loop_metrics(F, mavg64)
    step = np.linalg.norm(F[0] - F[1])
    assert abs(a["H_sw"] - b["H_sw"]) <= step * (1 + 1e-9)
    assert abs(a["M_r"] - b["M_r"]) <= 1e-3
    first = len(F)
    for mv in (mavg, mavg64):
        jump = np.nonzero(np.linalg.norm(np.diff(mv, axis=0), axis=1) > 0.02)[0]
        if len(jump):
            first = min(first, int(jump[0]) + 1)
    assert first > 40
    assert np.max(np.abs(mavg[:first] - mavg64[:first])) < 1e-3
    assert np.max(np.abs(np.linalg.norm(mm_.cpu().numpy(), axis=0) - 1)) < 1e-6
    # the float phase does the bulk of the iterations
    assert sum(r.heff_evals for r in rl) > sum(r.heff_evals for r in rh)


def test_mixed_rejects_mismatched_problems(mmlib):
    w = inputs.film_32x16x1()
    mat = mmlib.make_material(w.Ms, w.A, w.K)
    p64 = mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz), mat, mmlib.MM_FP64)
    p32 = mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, 8, w.nz, w.dx, w.dy, w.dz), mat, mmlib.MM_FP32)
    with pytest.raises(mmlib.MMError):
        mmlib.mm_hysteresis_sweep_mixed(p32, p64, dev(w.initial_m()), w.fields()[:3])
    with pytest.raises(mmlib.MMError):  # precisions swapped
        mmlib.mm_hysteresis_sweep_mixed(p64, p64, dev(w.initial_m()), w.fields()[:3])


def test_mixed_with_host_buffer_equals_device_buffer(mmlib):
    # m may live in host memory: it is staged through the FP64 problem's buffers
    w = inputs.film_32x16x1()
    grid = mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    mat = mmlib.make_material(w.Ms, w.A, w.K)
    p64 = mmlib.mm_setup_geometry(grid, mat, mmlib.MM_FP64)
    p32 = mmlib.mm_setup_geometry(grid, mat, mmlib.MM_FP32)
    F = w.fields()[:12]
    m_host = np.ascontiguousarray(w.initial_m())
    st_h, mavg_h, _, rh_h = mmlib.mm_hysteresis_sweep_mixed(p32, p64, m_host, F)
    m_dev = dev(w.initial_m())
    st_d, mavg_d, _, rh_d = mmlib.mm_hysteresis_sweep_mixed(p32, p64, m_dev, F)
    assert st_h == st_d == mmlib.MM_OK
    assert np.array_equal(mavg_h, mavg_d)
    assert np.array_equal(m_host, m_dev.cpu().numpy())
    assert [r.heff_evals for r in rh_h] == [r.heff_evals for r in rh_d]
