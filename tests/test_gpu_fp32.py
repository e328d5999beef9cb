"""FP32 field path (FFT and stencil arithmetic in float; tensor setup,
energies and step-size reductions in double) against the FP64 oracle.

Bars (stated per result): H_eff rel-L2 <= 3e-6 (a float FFT convolution of
this size carries ~1e-7 per element times its log depth); energy terms within
1e-5 of the largest term; a full 32x16x1 loop with the switching field within
one field step and the remanence within 1e-3, as for FP64."""
import numpy as np
import pytest
import torch

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs
from gpu_cases import dev, make_pair, rel_l2

pytestmark = pytest.mark.gpu
CELL = (3.90625e-9, 3.90625e-9, 5e-9)


@pytest.mark.parametrize("grid", [(1, 1, 1), (3, 2, 1), (7, 5, 3), (33, 17, 3), (128, 64, 2), (512, 256, 4)])
def test_heff_fp32(mmlib, grid):
    nx, ny, nz = grid
    prob, oprob = make_pair(mmlib, nx, ny, nz, CELL, precision=mmlib.MM_FP32)
    m = inputs.random_unit_m(oprob.shape, seed=5 + nx)
    Hext = np.array([1.0e4, 2.0e3, -3.0e3])
    H = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    mmlib.mm_heff(prob, dev(m, torch.float32), Hext, H)
    ref = om.heff(oprob, m.astype(np.float32).astype(np.float64), Hext, om.Demag(oprob))
    assert rel_l2(H.cpu().numpy(), ref) <= 3e-6


def test_energy_fp32(mmlib):
    prob, oprob = make_pair(mmlib, 40, 20, 2, CELL, K=2e4, precision=mmlib.MM_FP32)
    m = inputs.random_unit_m(oprob.shape, 9)
    E = mmlib.mm_energy(prob, dev(m, torch.float32), (4e3, 1e3, -2e3))
    ref = om.energy(oprob, m.astype(np.float32).astype(np.float64), (4e3, 1e3, -2e3), om.Demag(oprob))
    keys = ["demag", "exchange", "anisotropy", "zeeman", "total"]
    scale = max(abs(ref[k]) for k in keys)
    for i, k in enumerate(keys):
        assert abs(E[i] - ref[k]) <= 1e-5 * scale, (k, E[i], ref[k])


def test_full_loop_32x16x1_fp32(mmlib):
    w = inputs.film_32x16x1()
    prob, oprob = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K=w.K,
                            precision=mmlib.MM_FP32)
    F = w.fields()
    mavg_ref, _, _ = om.sweep(oprob, w.initial_m(), F, om.Demag(oprob), tol=w.tol)
    m = dev(w.initial_m(), torch.float32)
    st, mavg, res = mmlib.mm_hysteresis_sweep(prob, m, F, opts=mmlib.make_opts(tol=w.tol))
    assert st == mmlib.MM_OK
    a, b = om.loop_metrics(F, mavg), om.loop_metrics(F, mavg_ref)
    step = np.linalg.norm(F[0] - F[1])
    assert abs(a["H_sw"] - b["H_sw"]) <= step * (1 + 1e-9)
    assert abs(a["M_r"] - b["M_r"]) <= 1e-3
    norm_err = np.max(np.abs(np.linalg.norm(m.double().cpu().numpy(), axis=0) - 1))
    assert norm_err < 2e-5, norm_err
