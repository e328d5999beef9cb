"""Pins of the oracle's minimiser (Section 2) and hysteresis driver (Section 4).

* The closed-form step equals the numerical solution of the 3x3 linear
  midpoint system, Eq. (implicit_gradient_descent), and keeps |m| = 1.
* The step descends the energy for small tau.
* Barzilai-Borwein step sizes, Eq. (stepsize), on hand-built s, y, and the alternation.
* Stoner-Wohlfarth: a single cubic cell (isotropic demag, no exchange) switches
  at h_sw = (cos^(2/3) psi + sin^(2/3) psi)^(-3/2) H_K, within one field step.
"""
import math

import numpy as np
import pytest

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs


def test_cayley_step_solves_the_midpoint_system():
    prob = om.Problem(4, 3, 2, 3e-9, 3e-9, 3e-9, Ms=8e5, A=1.3e-11, K=500.0)
    m = inputs.random_unit_m(prob.shape, 2)
    H = om.heff(prob, m, (1e4, 0, 0), om.Demag(prob, workers=1))
    a = np.cross(m, H, axis=0)
    g = om.projected_gradient(m, H)
    tau = 3.7e-6
    m1 = om.cayley_step(m, g, tau)
    for idx in np.ndindex(prob.shape):
        ai = a[(slice(None),) + idx]
        mi = m[(slice(None),) + idx]
        Ax = np.array([[0, -ai[2], ai[1]], [ai[2], 0, -ai[0]], [-ai[1], ai[0], 0]])  # Ax v = a x v
        # descent orientation: m' = m - tau ((m+m')/2) x a  <=>  (I - tau/2 Ax) m' = (I + tau/2 Ax) m
        sol = np.linalg.solve(np.eye(3) - 0.5 * tau * Ax, (np.eye(3) + 0.5 * tau * Ax) @ mi)
        assert np.allclose(m1[(slice(None),) + idx], sol, rtol=0, atol=1e-14)
        # ... which is the printed scheme with its step parameter equal to -tau
        lhs = m1[(slice(None),) + idx]
        rhs = mi + (-tau) * np.cross(0.5 * (mi + lhs), ai)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-14)
    assert np.max(np.abs(np.linalg.norm(m1, axis=0) - 1)) < 1e-14


def test_projected_gradient_is_minus_tangential_field():
    m = inputs.random_unit_m((1, 2, 3), 8)
    H = inputs.random_unit_m((1, 2, 3), 9) * 1e5
    g = om.projected_gradient(m, H)
    mh = np.sum(m * H, axis=0)
    assert np.allclose(g, mh * m - H, rtol=0, atol=1e-9)
    assert np.max(np.abs(np.sum(g * m, axis=0))) < 1e-9


def test_small_step_descends_energy():
    prob = om.Problem(8, 4, 1, 5e-9, 5e-9, 5e-9, Ms=8e5, A=1.3e-11, K=500.0)
    d = om.Demag(prob, workers=1)
    m = inputs.random_unit_m(prob.shape, 3)
    Hext = (2e3, 1e3, 0.0)
    H = om.heff(prob, m, Hext, d)
    g = om.projected_gradient(m, H)
    E0 = om.energy(prob, m, Hext, d)["total"]
    for tau in (1e-9, 1e-8, 1e-2 / prob.Ms):
        for stepf in (om.cayley_step, om.normalize_step):
            assert om.energy(prob, stepf(m, g, tau), Hext, d)["total"] < E0


def test_bb_step_sizes_and_alternation():
    rng = np.random.default_rng(0)
    y = rng.standard_normal((3, 2, 2, 2))
    s = 0.25 * y
    assert math.isclose(om.bb_tau(1, s, y, 9.0), 0.25, rel_tol=1e-15)
    assert math.isclose(om.bb_tau(2, s, y, 9.0), 0.25, rel_tol=1e-15)
    s = rng.standard_normal((3, 2, 2, 2))
    y = s + 0.3 * rng.standard_normal((3, 2, 2, 2))
    ss, sy, yy = np.sum(s * s), np.sum(s * y), np.sum(y * y)
    assert om.bb_tau(3, s, y, 9.0) == ss / sy  # odd k: tau^1
    assert om.bb_tau(4, s, y, 9.0) == sy / yy  # even k: tau^2
    # non-positive curvature: |s|/|y|; nothing finite and positive: tau0
    assert math.isclose(om.bb_tau(1, s, -2.0 * s, 9.0), 0.5, rel_tol=1e-15)
    assert math.isclose(om.bb_tau(2, s, -2.0 * s, 9.0), 0.5, rel_tol=1e-15)
    assert om.bb_tau(2, s * 0, y * 0, 9.0) == 9.0
    assert om.bb_tau(1, s, y * 0, 9.0) == 9.0


def _sw_switching_field(psi_deg, step, tau_rule="alternate"):
    # One cubic cell: demag tensor is I/3, so H_d is parallel to m and exerts
    # no torque; without neighbours there is no exchange.  Uniaxial K along x.
    Ms, K = 8e5, 2.0e5
    prob = om.Problem(1, 1, 1, 4e-9, 4e-9, 4e-9, Ms=Ms, A=1.3e-11, K=K)
    HK = 2 * K / (om.MU0 * Ms)
    psi = math.radians(psi_deg)
    hdir = np.array([math.cos(psi), math.sin(psi), 0.0])
    hs = np.arange(1.2, -1.2, -step)
    d = om.Demag(prob, workers=1)
    m = np.zeros((3, 1, 1, 1)); m[0] = 1.0
    for h in hs:
        r = om.minimize(prob, m, h * HK * hdir, d, tol=1e-10, max_iter=20000, tau_rule=tau_rule)
        assert r.converged
        m = r.m
        if float(np.sum(m[:, 0, 0, 0] * hdir)) < 0:
            return h
    return None


@pytest.mark.parametrize("psi_deg,expect", [(1.0, None), (10.0, None), (30.0, None), (45.0, 0.5)])
def test_stoner_wohlfarth_switching_field(psi_deg, expect):
    psi = math.radians(psi_deg)
    hsw = (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** -1.5
    if expect is not None:
        assert math.isclose(hsw, expect, rel_tol=1e-12)
    if psi_deg == 1.0:
        assert abs(hsw - 0.90707) < 1e-5
    step = 0.002
    h = _sw_switching_field(psi_deg, step)
    assert h is not None
    # first field on the descending branch past the astroid: -hsw - step < h <= -hsw
    assert -hsw - step - 1e-9 < h <= -hsw + 1e-9


def test_minimize_small_film_converges_and_lowers_energy():
    w = inputs.film_32x16x1()
    prob = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K)
    d = om.Demag(prob, workers=1)
    m0 = inputs.random_unit_m(prob.shape, 1)
    Hext = w.fields()[30]
    r = om.minimize(prob, m0, Hext, d, tol=w.tol, max_iter=20000)
    assert r.converged and r.max_torque < w.tol and r.heff_evals == r.iters + 1
    assert om.energy(prob, r.m, Hext, d)["total"] < om.energy(prob, m0, Hext, d)["total"]
    assert np.max(np.abs(np.linalg.norm(r.m, axis=0) - 1)) < 1e-13
    H = om.heff(prob, r.m, Hext, d)
    assert om.max_torque(r.m, H, prob.Ms) == r.max_torque


def test_loop_metrics_on_a_synthetic_loop():
    H = inputs.sp1_sweep(5.0, 1.0, 0.0)
    h = H[:, 0]
    # <m_x> switches at -3 (descending) and +3 (ascending), remanence 0.9
    mx = np.where(np.arange(len(h)) < 11, np.where(h > -2.5 * 1e-3 / om.MU0, 0.9, -0.9), np.where(h < 2.5e-3 / om.MU0, -0.9, 0.9))
    mavg = np.stack([mx, np.zeros_like(mx), np.zeros_like(mx)], 1)
    r = om.loop_metrics(H, mavg)
    assert math.isclose(r["H_sw"], -3e-3 / om.MU0, rel_tol=1e-12)
    assert math.isclose(r["H_c"], -2.5e-3 / om.MU0, rel_tol=1e-12)
    assert r["M_r"] == 0.9


def test_normalize_step_returns_unit_vectors_along_the_explicit_step():
    """The renormalised explicit step, Eq. (projected_gradient_descent) in
    descent orientation: unit length even for steps far too large for the
    midpoint form, and parallel to m - tau g (a missing renormalisation, or
    a step taken along +g, fails here)."""
    m = inputs.random_unit_m((2, 3, 4), 21)
    H = inputs.random_unit_m((2, 3, 4), 22) * 7e5
    g = om.projected_gradient(m, H)
    for tau in (1e-9, 1e-6, 3e-6, 1e-3):
        m1 = om.normalize_step(m, g, tau)
        assert np.max(np.abs(np.linalg.norm(m1, axis=0) - 1.0)) < 1e-15
        v = m - tau * g
        assert np.max(np.abs(np.cross(m1, v, axis=0))) < 1e-12 * np.max(np.linalg.norm(v, axis=0))
        assert np.min(np.sum(m1 * v, axis=0)) > 0


def _sw_cell(psi_deg):
    Ms, K = 8e5, 2.0e5
    prob = om.Problem(1, 1, 1, 4e-9, 4e-9, 4e-9, Ms=Ms, A=1.3e-11, K=K)
    HK = 2 * K / (om.MU0 * Ms)
    psi = math.radians(psi_deg)
    return prob, HK, np.array([math.cos(psi), math.sin(psi), 0.0])


def test_sweep_opens_the_stoner_wohlfarth_loop_on_both_branches():
    """Section 4's driver on one cubic cell: descending then ascending
    branch.  The loop only opens (switching at -h_sw going down and +h_sw
    going up) if every field value starts from the previous magnetisation;
    restarting each value from the initial state would switch back at once
    on the ascending branch."""
    psi_deg = 30.0
    prob, HK, hdir = _sw_cell(psi_deg)
    psi = math.radians(psi_deg)
    hsw = (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** -1.5
    step = 0.004
    n = int(round(1.2 / step))
    h_desc = [1.2 - step * i for i in range(2 * n + 1)]
    h_asc = [-1.2 + step * i for i in range(1, 2 * n + 1)]
    hs = np.array(h_desc + h_asc)
    H_list = np.outer(hs * HK, hdir)
    m0 = np.zeros((3, 1, 1, 1)); m0[0] = 1.0
    mavg, res, mfin = om.sweep(prob, m0, H_list, om.Demag(prob, workers=1), tol=1e-10, max_iter=20000)
    assert all(r.converged for r in res)
    p = mavg @ hdir
    nd = len(h_desc)
    down = next(hs[i] for i in range(nd) if p[i] < 0)
    up = next(hs[i] for i in range(nd, len(hs)) if p[i] > 0)
    assert -hsw - step - 1e-9 < down <= -hsw + 1e-9
    assert hsw - 1e-9 <= up < hsw + step + 1e-9
    assert np.array_equal(mavg[-1], mfin.reshape(3, -1).mean(axis=1))


def test_sweep_is_a_chain_of_fresh_minimisations():
    """Per field value the sweep runs one minimisation from the previous
    result with the step-size history restarted (tau = tau0, k = 0); <m> is
    the mean of that result.  Replaying the chain with independent calls
    must give the same states, means and evaluation counts -- carrying tau
    or the BB history across field values changes the counts."""
    w = inputs.film_32x16x1()
    prob = om.Problem(8, 4, 1, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K)
    d = om.Demag(prob, workers=1)
    H_list = inputs.sp1_sweep(20.0, 10.0)[:4]          # +20, +10, 0, -10 mT
    m0 = inputs.tilted_uniform_m(prob.shape, 5)
    mavg, res, mfin = om.sweep(prob, m0, H_list, d, tol=1e-6, max_iter=5000)
    m = m0
    for j, H in enumerate(H_list):
        r = om.minimize(prob, m, H, d, tol=1e-6, max_iter=5000)
        m = r.m
        assert r.heff_evals == res[j].heff_evals and r.iters == res[j].iters
        assert r.converged and res[j].converged
        assert np.array_equal(mavg[j], m.reshape(3, -1).mean(axis=1))
        assert mavg[j][0] != m[0, 0, 0, 0]      # a mean over distinct cells, not one cell
    assert np.array_equal(m, mfin)
    # the first step of every field value uses tau0: a sweep over one value
    # equals a minimisation from the same state (no history to carry)
    mavg1, res1, _ = om.sweep(prob, mfin, H_list[:1], d, tol=1e-6, max_iter=5000)
    r1 = om.minimize(prob, mfin, H_list[0], d, tol=1e-6, max_iter=5000)
    assert res1[0].heff_evals == r1.heff_evals


def _pair(a, b):
    """s = (1, 0, 0), y = (a, b, 0) in one cell: s.s = 1, s.y = a, y.y = a^2 + b^2."""
    s = np.zeros((3, 1, 1, 1)); s[0] = 1.0
    y = np.zeros((3, 1, 1, 1)); y[0] = a; y[1] = b
    return s, y


def test_adaptive_switch_picks_by_the_angle_between_s_and_y():
    """Adaptive BB (Zhou, Gao and Dai 2006): short size tau^2 when
    (s.y)^2/((s.s)(y.y)) < kappa, else long size tau^1, whatever the parity of k."""
    s, y = _pair(2.0, 1.0)            # cos^2 = 4/5: long size 1/2
    for k in (1, 2, 3, 4):
        assert om.bb_tau(k, s, y, 9.0, "adaptive", 0.5) == 0.5
    s, y = _pair(1.0, 2.0)            # cos^2 = 1/5: short size 1/5
    for k in (1, 2, 3, 4):
        assert math.isclose(om.bb_tau(k, s, y, 9.0, "adaptive", 0.5), 0.2, rel_tol=1e-15)
    assert om.bb_tau(1, s, y, 9.0, "adaptive", 0.1) == 1.0      # cos^2 = 0.2 >= 0.1: long size 1/1
    s, y = _pair(-1.0, 1.0)           # negative curvature: |s|/|y| for both rules
    for rule in ("alternate", "adaptive"):
        assert math.isclose(om.bb_tau(2, s, y, 9.0, rule), 1 / math.sqrt(2), rel_tol=1e-15)


@pytest.mark.parametrize("rule", ["alternate", "adaptive"])
def test_bb_gradient_iteration_on_a_quadratic(rule):
    """f(x) = x^T A x / 2, A = diag(1 .. 100): for a quadratic y = A s, so
    both sizes are inverse Rayleigh quotients of A and lie in
    [1/lambda_max, 1/lambda_min]; the BB gradient iteration converges
    (Raydan, IMA J. Numer. Anal. 13 (1993) 321; the adaptive rule: Zhou, Gao
    and Dai 2006)."""
    lam = np.arange(1.0, 101.0).reshape(100, 1, 1, 1)
    x = np.ones((100, 1, 1, 1))
    g = lam * x
    x_prev = g_prev = None
    for k in range(400):
        if np.linalg.norm(g) < 1e-10 * np.sqrt(np.sum(lam ** 2)):
            break
        tau = 1e-2 if k == 0 else om.bb_tau(k, x - x_prev, g - g_prev, 1e-2, rule)
        assert 1 / 100 * (1 - 1e-12) <= tau <= 1.0 * (1 + 1e-12)
        x_prev, g_prev = x, g
        x = x - tau * g
        g = lam * x
    assert np.linalg.norm(g) < 1e-10 * np.sqrt(np.sum(lam ** 2)), (rule, k)


@pytest.mark.parametrize("psi_deg", [1.0, 30.0])
def test_stoner_wohlfarth_switching_with_the_adaptive_switch(psi_deg):
    psi = math.radians(psi_deg)
    hsw = (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** -1.5
    step = 0.002
    h = _sw_switching_field(psi_deg, step, tau_rule="adaptive")
    assert h is not None
    assert -hsw - step - 1e-9 < h <= -hsw + 1e-9
