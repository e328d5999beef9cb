"""Differentiation extension on the GPU (C ABI) against the CPU oracle.

* dU/dm = -mu0 Ms V H_eff (mm_energy_gradient, and torch autograd through
  Energy.apply) matches the oracle's field; the energy's directional finite
  difference matches the gradient.
* The tangent-plane Hessian-vector product matches the oracle's.
* The implicit adjoint d<m_x>/dK matches the oracle's adjoint at the oracle's
  converged minimum (small stiff film, where both CG solves converge tightly).
* At the 128x64x2 film (K_i uniform in [300, 700], relaxed at 0 mT from +x
  saturation at +50 mT)
  the adjoint matches central finite differences (dK = 1e-3 K) of <m_x> over
  re-minimisations on 32 random cells.  The bar is 1e-4 relative to the
  largest gradient entry: single entries range over five decades, and the
  smallest sit at the finite differences' noise floor."""
import numpy as np
import pytest
import torch

from oracle import micromag as om
from paper_1405_2728_gb300 import autograd, inputs
from gpu_cases import dev, make_pair, rel_l2

pytestmark = pytest.mark.gpu
CELL = (3.90625e-9, 3.90625e-9, 5e-9)


def test_energy_gradient_and_autograd(mmlib):
    prob, oprob = make_pair(mmlib, 24, 12, 2, CELL, K=3e4, u=(0.0, 0.6, 0.8))
    m0 = inputs.random_unit_m(oprob.shape, 31)
    Hext = (2e3, -1e3, 5e2)
    ref = -om.MU0 * oprob.Ms * oprob.V * om.heff(oprob, m0, Hext, om.Demag(oprob))
    G = torch.empty((3,) + oprob.shape, dtype=torch.float64, device="cuda")
    mmlib.mm_energy_gradient(prob, dev(m0), Hext, G)
    assert rel_l2(G.cpu().numpy(), ref) <= 1e-10
    m = dev(m0).requires_grad_(True)
    U = autograd.Energy.apply(m, prob, Hext)
    U.backward()
    assert rel_l2(m.grad.cpu().numpy(), ref) <= 1e-10
    # directional finite difference of the GPU energy along a random direction
    v = inputs.random_unit_m(oprob.shape, 32)
    h = 1e-6
    Ep = mmlib.mm_energy(prob, dev(m0 + h * v), Hext)[4]
    Em = mmlib.mm_energy(prob, dev(m0 - h * v), Hext)[4]
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - float(np.sum(ref * v))) <= 1e-7 * abs(fd)


def test_hessian_vec_matches_oracle(mmlib):
    prob, oprob = make_pair(mmlib, 20, 10, 3, CELL, K=5e3)
    m = inputs.random_unit_m(oprob.shape, 41)
    v = om.project(m, inputs.random_unit_m(oprob.shape, 42))
    Hext = (1e3, 0.0, 0.0)
    d = om.Demag(oprob)
    ref = om.hessian_vec(oprob, m, om.heff(oprob, m, Hext, d), v, d)
    Av = torch.empty((3,) + oprob.shape, dtype=torch.float64, device="cuda")
    mmlib.mm_hessian_vec(prob, dev(m), Hext, dev(v), Av)
    assert rel_l2(Av.cpu().numpy(), ref) <= 1e-10


def test_adjoint_matches_oracle_adjoint(mmlib):
    nx, ny, nz = 8, 4, 1
    cell = (5e-9, 5e-9, 5e-9)
    K = inputs.uniform(11, nx * ny * nz, 2e4, 6e4).reshape(nz, ny, nx)
    prob, oprob = make_pair(mmlib, nx, ny, nz, cell, K_cell=K)
    d = om.Demag(oprob)
    Hext = np.array([0.0, 2.0e4, 0.0])
    m0 = np.zeros((3, nz, ny, nx)); m0[0] = 1.0
    r = om.minimize(oprob, m0, Hext, d, tol=1e-12, max_iter=200000)
    assert r.converged
    dJdm = np.zeros_like(r.m); dJdm[0] = 1.0 / (nx * ny * nz)
    ref, _ = om.dJ_dK(oprob, r.m, Hext, dJdm, d, tol=1e-13)
    out = np.zeros((nz, ny, nx))
    st, it, res = mmlib.mm_adjoint_dK(prob, dev(r.m), Hext, dev(dJdm), out, tol=1e-13, max_iter=10000)
    assert st == mmlib.MM_OK and res < 1e-13
    assert np.max(np.abs(out - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_adjoint_matches_finite_differences_film_128x64x2(mmlib):
    w = inputs.film_128x64x2_random_K()
    K = w.K_cell
    prob, _ = make_pair(mmlib, w.nx, w.ny, w.nz, (w.dx, w.dy, w.dz), Ms=w.Ms, A=w.A, K_cell=K)
    # from +x saturation: minimise at +50 mT (tilted 1 degree toward +y, as in
    # the sweeps, which breaks the transverse symmetry) and then at 0 mT
    m = dev(w.initial_m())
    st, r = mmlib.mm_minimize(prob, m, w.fields()[0], mmlib.make_opts(tol=1e-10, max_iter=400000))
    assert st == mmlib.MM_OK
    tight = mmlib.make_opts(tol=1e-14, max_iter=400000)
    st, r = mmlib.mm_minimize(prob, m, (0, 0, 0), tight)
    assert st == mmlib.MM_OK
    g, st, it = autograd.dmx_dK(prob, m, (0, 0, 0), tol=1e-11, max_iter=200000)
    assert st == mmlib.MM_OK
    g = g.cpu().numpy()
    cells = inputs.splitmix64(2728, 32) % np.uint64(w.ncells)
    worst = 0.0
    for c in cells.astype(np.int64):
        idx = np.unravel_index(c, w.shape)
        dK = 1e-3 * K[idx]
        vals = []
        for sgn in (1, -1):
            Kp = K.copy(); Kp[idx] += sgn * dK
            mmlib.mm_set_anisotropy(prob, Kp)
            mp = m.clone()
            st, _ = mmlib.mm_minimize(prob, mp, (0, 0, 0), tight)
            assert st == mmlib.MM_OK
            vals.append(float(mp[0].mean()))
        fd = (vals[0] - vals[1]) / (2 * dK)
        worst = max(worst, abs(fd - g[idx]))
    mmlib.mm_set_anisotropy(prob, K)
    assert worst <= 1e-4 * np.max(np.abs(g)), (worst, np.max(np.abs(g)))
