"""Pins of the oracle's implicit adjoint (differentiation extension).

* Single cubic cell (isotropic demag, no exchange) in an in-plane field at
  angle psi: the equilibrium angle obeys K sin 2t = mu0 Ms H sin(psi - t), so
  d<m_x>/dK = -sin t * dt/dK with dt/dK = -sin 2t / (2K cos 2t + mu0 Ms H cos(psi - t)).
* A small film: central finite differences of <m_x> over re-minimisations
  with K_i +- dK agree with the adjoint gradient.
* A is symmetric on tangent fields (the adjoint relies on it)."""
import math

import numpy as np
import pytest

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs


def test_single_cell_closed_form():
    Ms, K = 8e5, 2e4
    prob = om.Problem(1, 1, 1, 4e-9, 4e-9, 4e-9, Ms=Ms, A=1.3e-11, K=K)
    d = om.Demag(prob, workers=1)
    psi = math.radians(30.0)
    Hmag = 0.3 * 2 * K / (om.MU0 * Ms)
    Hext = Hmag * np.array([math.cos(psi), math.sin(psi), 0.0])
    m0 = np.array([1.0, 0.0, 0.0]).reshape(3, 1, 1, 1)
    r = om.minimize(prob, m0, Hext, d, tol=1e-13, max_iter=100000)
    assert r.converged
    t = math.atan2(r.m[1, 0, 0, 0], r.m[0, 0, 0, 0])
    assert abs(K * math.sin(2 * t) - om.MU0 * Ms * Hmag * math.sin(psi - t)) < 1e-6 * K
    dtdK = -math.sin(2 * t) / (2 * K * math.cos(2 * t) + om.MU0 * Ms * Hmag * math.cos(psi - t))
    expect = -math.sin(t) * dtdK
    dJdm = np.zeros((3, 1, 1, 1)); dJdm[0] = 1.0
    g, _ = om.dJ_dK(prob, r.m, Hext, dJdm, d)
    assert abs(g[0, 0, 0] - expect) <= 1e-9 * abs(expect)


def test_operator_is_symmetric_on_tangent_fields():
    prob = om.Problem(6, 4, 2, 4e-9, 4e-9, 5e-9, Ms=8e5, A=1.3e-11, K=inputs.uniform(3, 48, 300, 700).reshape(2, 4, 6))
    d = om.Demag(prob, workers=1)
    m = inputs.random_unit_m(prob.shape, 4)
    H = om.heff(prob, m, (1e3, 0, 0), d)
    a = om.project(m, inputs.random_unit_m(prob.shape, 5))
    b = om.project(m, inputs.random_unit_m(prob.shape, 6))
    lhs = np.sum(a * om.hessian_vec(prob, m, H, b, d))
    rhs = np.sum(b * om.hessian_vec(prob, m, H, a, d))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_small_film_matches_finite_differences():
    nx, ny, nz = 8, 4, 1
    K = inputs.uniform(11, nx * ny * nz, 2e4, 6e4).reshape(nz, ny, nx)
    prob = om.Problem(nx, ny, nz, 5e-9, 5e-9, 5e-9, Ms=8e5, A=1.3e-11, K=K)
    d = om.Demag(prob, workers=1)
    Hext = np.array([0.0, 2.0e4, 0.0])
    m0 = np.zeros((3, nz, ny, nx)); m0[0] = 1.0
    r = om.minimize(prob, m0, Hext, d, tol=1e-12, max_iter=200000)
    assert r.converged
    dJdm = np.zeros_like(r.m); dJdm[0] = 1.0 / (nx * ny * nz)
    g, _ = om.dJ_dK(prob, r.m, Hext, dJdm, d)
    for idx in [(0, 0, 0), (0, 2, 5), (0, 3, 7), (0, 1, 3)]:
        dK = 1e-3 * K[idx]
        vals = []
        for sgn in (1, -1):
            Kp = K.copy(); Kp[idx] += sgn * dK
            pp = om.Problem(nx, ny, nz, 5e-9, 5e-9, 5e-9, Ms=8e5, A=1.3e-11, K=Kp)
            rp = om.minimize(pp, r.m, Hext, d, tol=1e-12, max_iter=200000)
            assert rp.converged
            vals.append(rp.m[0].mean())
        fd = (vals[0] - vals[1]) / (2 * dK)
        assert abs(fd - g[idx]) <= 1e-4 * np.max(np.abs(g)), (idx, fd, g[idx])
