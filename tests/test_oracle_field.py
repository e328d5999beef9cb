"""Pins of the oracle's effective field and energy.

* FFT demag equals the direct O(N^2) sum with the same tensor (tiny and ragged grids).
* Uniform magnetisation: the mean demag field is -Ms N_body m (body-sum identity).
* Exchange: zero for uniform m; the closed form of a planar spiral.
* Every term: H_i = -(1/(mu0 Ms V)) dU/dm_i by central finite differences of
  the separately coded energy (pins the 1/2 of the demag energy, factors of 2
  and signs of every term).
"""
import math

import numpy as np
import pytest

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs


def _prob(nx, ny, nz, cell=(3.0e-9, 4.0e-9, 5.0e-9), K=500.0, u=(1.0, 0.0, 0.0)):
    return om.Problem(nx, ny, nz, *cell, Ms=8.0e5, A=1.3e-11, K=K, u=u)


@pytest.mark.parametrize("grid", [(1, 1, 1), (2, 1, 1), (1, 3, 1), (3, 2, 1), (2, 2, 2), (5, 3, 2), (7, 5, 3), (4, 1, 6)])
def test_fft_demag_equals_direct_sum(grid):
    prob = _prob(*grid)
    m = inputs.random_unit_m(prob.shape, seed=11 + sum(grid))
    full = om.newell_full(prob)
    d = om.Demag(prob, full, workers=1)
    Hf = d.field(m)
    Hd = om.demag_direct(prob, m, full)
    assert np.linalg.norm(Hf - Hd) <= 1e-13 * np.linalg.norm(Hd)


def test_sampled_direct_cells_match_full_direct():
    prob = _prob(6, 4, 3)
    m = inputs.random_unit_m(prob.shape, seed=3)
    full = om.newell_full(prob)
    Hd = om.demag_direct(prob, m, full)
    cells = [0, 5, 17, 40, 71]
    Hs = om.demag_direct(prob, m, full, cells=cells)
    assert np.allclose(Hs, Hd.reshape(3, -1)[:, cells], rtol=0, atol=1e-9)


def test_uniform_m_mean_demag_is_body_factor():
    prob = _prob(6, 5, 2)
    mdir = np.array([0.6, -0.48, 0.64])
    m = np.broadcast_to(mdir.reshape(3, 1, 1, 1), (3,) + prob.shape).copy()
    H = om.Demag(prob, workers=1).field(m)
    Nb = om.newell_entry(0, 0, 0, prob.nx * prob.dx, prob.ny * prob.dy, prob.nz * prob.dz)
    Nmat = np.array([[Nb[0], Nb[3], Nb[4]], [Nb[3], Nb[1], Nb[5]], [Nb[4], Nb[5], Nb[2]]])
    mean = H.reshape(3, -1).mean(axis=1)
    assert np.allclose(mean, -prob.Ms * Nmat @ mdir, rtol=1e-12, atol=1e-9)


def test_exchange_vanishes_for_uniform_m():
    prob = _prob(6, 4, 3)
    m = np.zeros((3,) + prob.shape)
    m[2] = 1.0
    assert np.all(om.exchange_field(prob, m) == 0)
    assert om.energy(prob, m, (0, 0, 0), om.Demag(prob, workers=1))["exchange"] == 0.0


def test_exchange_spiral_closed_form():
    nx, ny, nz = 16, 3, 2
    prob = _prob(nx, ny, nz, K=0.0)
    q = 0.3  # rotation per cell (rad)
    ang = q * np.arange(nx)
    m = np.zeros((3,) + prob.shape)
    m[0] = np.cos(ang)[None, None, :]
    m[1] = np.sin(ang)[None, None, :]
    E = om.energy(prob, m, (0, 0, 0), om.Demag(prob, workers=1))["exchange"]
    expect = prob.A * prob.V * (nx - 1) * ny * nz * (2 - 2 * math.cos(q)) / prob.dx**2
    assert abs(E - expect) <= 1e-13 * expect
    H = om.exchange_field(prob, m)
    c = 2 * prob.A / (om.MU0 * prob.Ms) * (2 * math.cos(q) - 2) / prob.dx**2
    assert np.allclose(H[:, :, :, 1:-1], c * m[:, :, :, 1:-1], rtol=1e-12, atol=1e-6)


def test_anisotropy_and_zeeman_closed_forms():
    prob = _prob(2, 2, 1, K=1234.0, u=(0.0, 0.6, 0.8))
    m = inputs.random_unit_m(prob.shape, 5)
    Ha = om.anisotropy_field(prob, m)
    mu = 0.6 * m[1] + 0.8 * m[2]
    assert np.allclose(Ha[1], 2 * 1234.0 / (om.MU0 * prob.Ms) * mu * 0.6, rtol=1e-14)
    E = om.energy(prob, m, (100.0, -50.0, 7.0), om.Demag(prob, workers=1))
    assert abs(E["anisotropy"] - np.sum(1234.0 * prob.V * (1 - mu**2))) < 1e-14 * abs(E["anisotropy"])
    zexp = -om.MU0 * prob.Ms * prob.V * np.sum(100.0 * m[0] - 50.0 * m[1] + 7.0 * m[2])
    assert abs(E["zeeman"] - zexp) < 1e-14 * abs(zexp)


@pytest.mark.parametrize("percell", [False, True])
def test_field_is_energy_gradient(percell):
    # H_i = -(1/(mu0 Ms V)) dU/dm_i, checked by central differences of U.
    prob = _prob(5, 4, 2, K=3.0e4)
    if percell:
        prob.K = inputs.uniform(9, 40, 1e4, 5e4).reshape(prob.shape)
        u = inputs.random_unit_m(prob.shape, 21)
        prob.u = u
    m = inputs.random_unit_m(prob.shape, 4)
    Hext = np.array([2.0e4, -1.0e4, 5.0e3])
    d = om.Demag(prob, workers=1)
    H = om.heff(prob, m, Hext, d)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        a, k, j, i = rng.integers(3), rng.integers(prob.nz), rng.integers(prob.ny), rng.integers(prob.nx)
        mp = m.copy(); mp[a, k, j, i] += h
        mm = m.copy(); mm[a, k, j, i] -= h
        dU = (om.energy(prob, mp, Hext, d)["total"] - om.energy(prob, mm, Hext, d)["total"]) / (2 * h)
        Hfd = -dU / (om.MU0 * prob.Ms * prob.V)
        assert abs(Hfd - H[a, k, j, i]) <= 1e-7 * np.max(np.abs(H))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_uniform_cube_demag_energy_is_one_sixth(n):
    # A uniformly magnetised cube has the body demagnetising factor 1/3 along
    # every direction, so its demag energy is mu0 Ms^2 L^3 / 6 for any m,
    # whatever the number of cells.
    a = 4.0e-9
    prob = om.Problem(n, n, n, a, a, a, Ms=8.0e5, A=1.3e-11, K=0.0)
    for mdir in ([1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.48, -0.6, 0.64]):
        m = np.broadcast_to(np.reshape(mdir, (3, 1, 1, 1)), (3,) + prob.shape).copy()
        E = om.energy(prob, m, (0, 0, 0), om.Demag(prob, workers=1))["demag"]
        expect = om.MU0 * prob.Ms**2 * (n * a) ** 3 / 6.0
        assert abs(E - expect) <= 1e-12 * expect


@pytest.mark.parametrize("mdir,factor", [((1.0, 0.0, 0.0), -2.0), ((0.0, 1.0, 0.0), 1.0), ((0.0, 0.0, 1.0), 1.0)])
def test_two_distant_cells_interact_as_point_dipoles(mdir, factor):
    # Two cubic cells R apart along x, the cells between them empty (m = 0).
    # E_d = two self energies (mu0 Ms^2 V / 6 each) plus the dipole-dipole
    # energy mu0 Ms^2 V^2 (m1.m2 - 3 (m1.x)(m2.x)) / (4 pi R^3).  For cubes the
    # first correction to the point dipole is of order (a/R)^4 (6.7e-6 here).
    a, R = 5.0e-9, 16
    prob = om.Problem(R + 1, 1, 1, a, a, a, Ms=8.0e5, A=1.3e-11, K=0.0)
    m = np.zeros((3,) + prob.shape)
    m[:, 0, 0, 0] = mdir
    m[:, 0, 0, R] = mdir
    E = om.energy(prob, m, (0, 0, 0), om.Demag(prob, workers=1))["demag"]
    V = a**3
    self_e = 2 * om.MU0 * prob.Ms**2 * V / 6.0
    dip = om.MU0 * prob.Ms**2 * V * V * factor / (4 * math.pi * (R * a) ** 3)
    assert abs((E - self_e) - dip) <= 2e-5 * abs(dip)


@pytest.mark.parametrize("axis", ["y", "z"])
def test_exchange_spiral_along_y_and_z(axis):
    # The spiral closed form along each of the other axes, with cell sizes
    # that differ per axis (3, 4, 5 nm): catches a cell size taken from the
    # wrong axis, which the energy-gradient check alone would not.
    q = 0.25
    shape = {"y": (2, 12, 3), "z": (3, 2, 10)}[axis]  # nx, ny, nz
    prob = _prob(*shape, K=0.0)
    n_ax, d, ax = {"y": (shape[1], prob.dy, 2), "z": (shape[2], prob.dz, 1)}[axis]
    ang = q * np.arange(n_ax)
    m = np.zeros((3,) + prob.shape)
    bshape = [1, 1, 1]
    bshape[ax - 1] = n_ax
    m[0] = np.broadcast_to(np.cos(ang).reshape(bshape), prob.shape)
    m[2] = np.broadcast_to(np.sin(ang).reshape(bshape), prob.shape)
    E = om.energy(prob, m, (0, 0, 0), om.Demag(prob, workers=1))["exchange"]
    bonds = prob.nx * prob.ny * prob.nz // n_ax * (n_ax - 1)
    expect = prob.A * prob.V * bonds * (2 - 2 * math.cos(q)) / d**2
    assert abs(E - expect) <= 1e-13 * expect
    H = om.exchange_field(prob, m)
    c = 2 * prob.A / (om.MU0 * prob.Ms) * (2 * math.cos(q) - 2) / d**2
    inner = [slice(None)] * 4
    inner[ax] = slice(1, -1)
    assert np.allclose(H[tuple(inner)], c * m[tuple(inner)], rtol=1e-12, atol=1e-6)
