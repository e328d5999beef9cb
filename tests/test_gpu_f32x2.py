"""Double-float precision (MM_F32X2, an extension): the caller's arrays in
double; the iterates, the FFTs, the demagnetisation convolution, the local
terms, the step and the per-CTA sums in pairs of floats (about 48
significant bits); the sums across CTAs and the step size in double.

Bars.  H_eff against the FP64 oracle: rel-L2 <= 1e-10, the FP64 target (the
double-float FFT carries ~1e-14 per element times its log depth).  Energy
terms within 1e-11 of the largest term.  Minimiser steps from the oracle's
start: the per-evaluation field error is ~100 times that of FP64, so the
25-step trajectory bar is 1e-7 rel-L2 (FP64: 1e-8), and the whole
32 x 16 x 1 loop as for FP64 (switching field within one field step,
remanence within 1e-3).  Grids that need the bulk layout are refused."""
import numpy as np
import pytest
import torch

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs
from gpu_cases import dev, make_pair, rel_l2

pytestmark = pytest.mark.gpu
CELL = (3.90625e-9, 3.90625e-9, 5e-9)


@pytest.mark.parametrize("grid", [(1, 1, 1), (3, 2, 1), (7, 5, 3), (16, 8, 2), (33, 17, 3), (32, 16, 1),
                                  (9, 40, 4), (128, 64, 2), (512, 256, 4)])
def test_heff_f32x2_matches_oracle(mmlib, grid):
    nx, ny, nz = grid
    prob, oprob = make_pair(mmlib, nx, ny, nz, CELL, precision=mmlib.MM_F32X2)
    m = inputs.random_unit_m(oprob.shape, seed=300 + nx + 7 * ny + 31 * nz)
    Hext = np.array([1.5e4, -7.0e3, 2.0e3])
    H = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    mmlib.mm_heff(prob, dev(m), Hext, H)
    ref = om.heff(oprob, m, Hext, om.Demag(oprob))
    err = rel_l2(H.cpu().numpy(), ref)
    print("f32x2 H_eff rel-L2", grid, err)
    assert err <= 1e-10


def test_energy_f32x2(mmlib):
    prob, oprob = make_pair(mmlib, 40, 20, 2, CELL, K=2e4, precision=mmlib.MM_F32X2)
    m = inputs.random_unit_m(oprob.shape, 9)
    E = mmlib.mm_energy(prob, dev(m), (4e3, 1e3, -2e3))
    ref = om.energy(oprob, m, (4e3, 1e3, -2e3), om.Demag(oprob))
    keys = ["demag", "exchange", "anisotropy", "zeeman", "total"]
    scale = max(abs(ref[k]) for k in keys)
    for i, k in enumerate(keys):
        assert abs(E[i] - ref[k]) <= 1e-11 * scale, (k, E[i], ref[k])


def test_f32x2_per_cell_material(mmlib):
    """Per-cell K and easy axes stay double and enter the double-word local
    terms converted per load: the field (host buffers, staged by the library),
    the energies and 25 minimiser steps against the oracle."""
    nx, ny, nz = 24, 12, 3
    shape = (nz, ny, nx)
    K = inputs.uniform(3, nx * ny * nz, 1e3, 5e4).reshape(shape)
    u = inputs.random_unit_m(shape, 17)
    prob, oprob = make_pair(mmlib, nx, ny, nz, CELL, K_cell=K, u_cell=u, precision=mmlib.MM_F32X2)
    m = inputs.random_unit_m(shape, 18)
    H = np.zeros((3,) + shape)
    mmlib.mm_heff(prob, m, (0.0, 3e3, 0.0), H)
    demag = om.Demag(oprob)
    assert rel_l2(H, om.heff(oprob, m, (0.0, 3e3, 0.0), demag)) <= 1e-10
    E = mmlib.mm_energy(prob, dev(m), (0.0, 3e3, 0.0))
    ref = om.energy(oprob, m, (0.0, 3e3, 0.0), demag)
    keys = ["demag", "exchange", "anisotropy", "zeeman", "total"]
    scale = max(abs(ref[k]) for k in keys)
    for i, k in enumerate(keys):
        assert abs(E[i] - ref[k]) <= 1e-11 * scale, (k, E[i], ref[k])
    mg = dev(m)
    st, r = mmlib.mm_minimize(prob, mg, (0.0, 3e3, 0.0), mmlib.make_opts(tol=0.0, max_iter=25))
    assert st == mmlib.MM_ERR_NOT_CONVERGED and r.iters == 25
    ref_m = om.minimize(oprob, m, (0.0, 3e3, 0.0), demag, tol=0.0, max_iter=25).m
    assert rel_l2(mg.cpu().numpy(), ref_m) <= 1e-7


def test_f32x2_inspect_returns_the_iterates_and_their_sums(mmlib):
    """mm_min_inspect on a double-word problem: the iterates and gradients
    come back as the double nearest to each pair (m_k equal to what the
    minimisation returned), and the step-size sums of Eq. (stepsize), formed
    by the kernels in double-word arithmetic, agree with a float64 reduction
    of those doubles (their rounding to double moves s and y by ~1e-16 of m)."""
    w = inputs.film_128x64x2()
    prob, _ = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K=w.K,
                        precision=mmlib.MM_F32X2)
    m = dev(w.initial_m())
    mmlib.mm_minimize(prob, m, w.fields()[30], mmlib.make_opts(tol=0.0, max_iter=12))
    bufs = [torch.empty(prob.shape, dtype=torch.float64, device="cuda") for _ in range(4)]
    stt = mmlib.mm_min_inspect(prob, *bufs)
    assert stt["k"] == 12
    mk, mp, gk, gp = (b.cpu().numpy() for b in bufs)
    assert np.array_equal(mk, m.cpu().numpy())
    assert np.max(np.abs(np.linalg.norm(mk, axis=0) - 1)) < 1e-13
    s_, y_ = mk - mp, gk - gp
    ss, sy, yy = float(np.sum(s_ * s_)), float(np.sum(s_ * y_)), float(np.sum(y_ * y_))
    assert abs(stt["ss"] - ss) <= 1e-8 * ss
    assert abs(stt["yy"] - yy) <= 1e-8 * yy
    assert abs(stt["sy"] - sy) <= 1e-8 * np.sqrt(ss * yy)


@pytest.mark.parametrize("step", [0, 1])
def test_fixed_steps_f32x2_follow_the_oracle(mmlib, step):
    w = inputs.film_32x16x1()
    prob, oprob = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K=w.K,
                            precision=mmlib.MM_F32X2)
    m0 = inputs.random_unit_m(oprob.shape, 21)
    H = w.fields()[40]
    m = dev(m0)
    st, r = mmlib.mm_minimize(prob, m, H, mmlib.make_opts(tol=0.0, max_iter=25, step_kind=step))
    assert st == mmlib.MM_ERR_NOT_CONVERGED and r.iters == 25
    ref = om.minimize(oprob, m0, H, om.Demag(oprob), tol=0.0, max_iter=25,
                      step="cayley" if step == 0 else "normalize")
    err = rel_l2(m.cpu().numpy(), ref.m)
    print("f32x2 25 steps rel-L2", err)
    assert err <= 1e-7
    assert np.max(np.abs(np.linalg.norm(m.cpu().numpy(), axis=0) - 1)) < 25 * 1e-14


def test_fixed_steps_f32x2_at_512x256x4(mmlib):
    w = inputs.film_512x256x4()
    prob, oprob = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K=w.K,
                            precision=mmlib.MM_F32X2)
    assert mmlib.mm_problem_info(prob)["precision"] == mmlib.MM_F32X2
    m = dev(w.initial_m())
    st, r = mmlib.mm_minimize(prob, m, w.fields()[60], mmlib.make_opts(tol=0.0, max_iter=25))
    assert st == mmlib.MM_ERR_NOT_CONVERGED and r.iters == 25
    ref = om.minimize(oprob, w.initial_m(), w.fields()[60], om.Demag(oprob), tol=0.0, max_iter=25)
    err = rel_l2(m.cpu().numpy(), ref.m)
    print("f32x2 512x256x4 25 steps rel-L2", err)
    assert err <= 1e-7
    assert abs(r.max_torque - ref.max_torque) <= 1e-6 * ref.max_torque


def test_full_loop_32x16x1_f32x2(mmlib):
    w = inputs.film_32x16x1()
    prob, oprob = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K=w.K,
                            precision=mmlib.MM_F32X2)
    F = w.fields()
    mavg_ref, res_ref, _ = om.sweep(oprob, w.initial_m(), F, om.Demag(oprob), tol=w.tol)
    m = dev(w.initial_m())
    st, mavg, res = mmlib.mm_hysteresis_sweep(prob, m, F, opts=mmlib.make_opts(tol=w.tol))
    assert st == mmlib.MM_OK and all(r.converged for r in res)
    a, b = om.loop_metrics(F, mavg), om.loop_metrics(F, mavg_ref)
    step = np.linalg.norm(F[0] - F[1])
    assert abs(a["H_sw"] - b["H_sw"]) <= step * (1 + 1e-9)
    assert abs(a["M_r"] - b["M_r"]) <= 1e-3
    evals = sum(r.heff_evals for r in res)
    evals_ref = sum(r.heff_evals for r in res_ref)
    assert abs(evals - evals_ref) <= 0.2 * evals_ref


def test_bulk_grids_are_refused(mmlib):
    with pytest.raises(mmlib.MMError) as e:
        mmlib.mm_setup_geometry(mmlib.make_grid(8, 8, 8, *CELL), mmlib.make_material(8e5, 1.3e-11, 500.0),
                                mmlib.MM_F32X2)
    assert e.value.status == mmlib.MM_ERR_UNSUPPORTED
