"""Pins of the oracle's Newell tensor against facts it must satisfy.

None of these re-types the oracle's formula: the trace rule, the point-dipole
far field, sub-cell quadrature of the dipole kernel, the body-sum identity and
Aharoni's closed-form prism demagnetising factor are independent of Newell's
f and g, so a dropped term, a wrong weight, sign or permutation fails one.
"""
import math

import mpmath
import numpy as np
import pytest

from oracle import micromag as om

CELLS = [(1.0, 1.0, 1.0), (1.0, 2.0, 0.5), (3.90625, 3.90625, 5.0), (31.25, 31.25, 20.0), (2.0, 1.0, 1.0)]


def test_quad_type_is_binary128():
    assert om._lib().oracle_quad_mant_dig() >= 113


@pytest.mark.parametrize("cell", CELLS)
def test_trace_is_one_at_origin(cell):
    N = om.newell_entry(0, 0, 0, *cell)
    assert abs(N[:3].sum() - 1.0) < 4e-16
    assert np.all(N[:3] > 0)
    assert np.all(np.abs(N[3:]) < 1e-15)


def test_cube_self_term_is_one_third():
    N = om.newell_entry(0, 0, 0, 2.5, 2.5, 2.5)
    assert np.allclose(N[:3], 1.0 / 3.0, rtol=0, atol=2e-16)


@pytest.mark.parametrize("off", [(1, 0, 0), (2, 1, 0), (7, 5, 3), (64, 3, 1), (511, 255, 3), (1000, 7, 2)])
@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (3.90625, 3.90625, 5.0)])
def test_trace_vanishes_off_origin(off, cell):
    # Laplace: outside the source cell the trace of the demag kernel is 0.
    # At R ~ 1000 cells the 27-point difference cancels ~1e18 of f; only the
    # quad evaluation keeps this at rounding level.
    N = om.newell_entry(*off, *cell)
    scale = np.max(np.abs(N[:3]))
    assert abs(N[:3].sum()) <= 1e-13 * scale


def _dipole(off, cell):
    r = np.array(off, float) * np.array(cell)
    R = np.linalg.norm(r)
    V = np.prod(cell)
    D = -(V / (4 * math.pi)) * (3 * np.outer(r, r) / R**2 - np.eye(3)) / R**3
    return np.array([D[0, 0], D[1, 1], D[2, 2], D[0, 1], D[0, 2], D[1, 2]])


@pytest.mark.parametrize("cell", [(1.0, 2.0, 0.5), (3.90625, 3.90625, 5.0)])
@pytest.mark.parametrize("direction", [(3, 2, 1), (-2, 5, 3), (4, -1, -3)])
def test_far_field_is_point_dipole(cell, direction):
    # N -> -(V/4pi)(3 rr^T/r^2 - I)/r^3 with relative error O((d/R)^2).
    # Oblique directions make every component non-zero, which pins signs
    # and the permutation of the off-diagonal entries.
    errs = []
    for scale in (20, 40, 80):
        off = tuple(scale * d for d in direction)
        N = om.newell_entry(*off, *cell)
        D = _dipole(off, cell)
        errs.append(np.max(np.abs(N - D)) / np.max(np.abs(D)))
    assert errs[-1] < 2e-4
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0  # second-order convergence


def _subcell_dipole_average(off, cell, s):
    """Average of the point-dipole kernel over s^3 x s^3 midpoint sub-cell pairs."""
    cell = np.array(cell)
    g = (np.arange(s) + 0.5) / s - 0.5
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * cell
    d = np.array(off, float) * cell
    r = (d + P[:, None, :] - P[None, :, :]).reshape(-1, 3)
    R2 = np.sum(r * r, 1)
    R = np.sqrt(R2)
    V = np.prod(cell)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    out = []
    for a, b in pairs:
        k = (3 * r[:, a] * r[:, b] / R2 - (a == b)) / R**3
        out.append(-(V / (4 * math.pi)) * k.mean())
    return np.array(out)


@pytest.mark.parametrize("off", [(2, 1, 0), (2, 2, 1), (0, 3, 2)])
def test_near_field_matches_subcell_dipole_quadrature(off):
    # For non-touching cells the Newell tensor is the pair average of the
    # dipole kernel; the midpoint rule converges as 1/s^2 (Richardson).
    cell = (1.0, 1.3, 0.7)
    N = om.newell_entry(*off, *cell)
    a4 = _subcell_dipole_average(off, cell, 4)
    a8 = _subcell_dipole_average(off, cell, 8)
    extrap = (4 * a8 - a4) / 3
    scale = np.max(np.abs(N))
    assert np.max(np.abs(extrap - N)) < 2e-4 * scale
    assert np.max(np.abs(a8 - N)) < np.max(np.abs(a4 - N))


def _aharoni_Dz(a, b, c):
    """Aharoni (J. Appl. Phys. 83, 3432, 1998): magnetometric demagnetising
    factor along z of a 2a x 2b x 2c prism, in multiprecision."""
    a, b, c = mpmath.mpf(a), mpmath.mpf(b), mpmath.mpf(c)
    r = mpmath.sqrt(a * a + b * b + c * c)
    ab = mpmath.sqrt(a * a + b * b)
    bc = mpmath.sqrt(b * b + c * c)
    ac = mpmath.sqrt(a * a + c * c)
    ln = mpmath.log
    t = ((b * b - c * c) / (2 * b * c) * ln((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * ln((r - b) / (r + b))
         + b / (2 * c) * ln((ab + a) / (ab - a))
         + a / (2 * c) * ln((ab + b) / (ab - b))
         + c / (2 * a) * ln((bc - b) / (bc + b))
         + c / (2 * b) * ln((ac - a) / (ac + a))
         + 2 * mpmath.atan(a * b / (c * r))
         + (a**3 + b**3 - 2 * c**3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab**3 + bc**3 + ac**3) / (3 * a * b * c))
    return t / mpmath.pi


@pytest.mark.parametrize("cell", [(1.0, 2.0, 0.5), (3.90625, 3.90625, 5.0), (31.25, 31.25, 20.0), (7.0, 1.0, 3.0)])
def test_self_term_equals_aharoni_prism_factor(cell):
    mpmath.mp.dps = 40
    a, b, c = (x / 2 for x in cell)
    Dx, Dy, Dz = float(_aharoni_Dz(b, c, a)), float(_aharoni_Dz(c, a, b)), float(_aharoni_Dz(a, b, c))
    assert abs(Dx + Dy + Dz - 1.0) < 1e-15  # the closed form's own sum rule
    N = om.newell_entry(0, 0, 0, *cell)
    assert np.allclose(N[:3], [Dx, Dy, Dz], rtol=0, atol=1e-15)


@pytest.mark.parametrize("grid", [(5, 3, 2), (8, 4, 1), (3, 3, 3)])
def test_body_sum_identity(grid):
    # (1/Ncells) sum_i sum_j N(r_i - r_j) equals the self factor of one
    # cuboid the size of the whole body (the pair average over the body).
    nx, ny, nz = grid
    cell = (1.0, 1.5, 0.8)
    full = om.newell_full(om.Problem(nx, ny, nz, *cell, Ms=1.0, A=0.0))
    cnt = (np.array([nz - abs(k) for k in range(-(nz - 1), nz)])[:, None, None]
           * np.array([ny - abs(j) for j in range(-(ny - 1), ny)])[None, :, None]
           * np.array([nx - abs(i) for i in range(-(nx - 1), nx)])[None, None, :])
    lhs = np.array([np.sum(full[c] * cnt) for c in range(6)]) / (nx * ny * nz)
    rhs = om.newell_entry(0, 0, 0, nx * cell[0], ny * cell[1], nz * cell[2])
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-14)


def test_octant_matches_direct_entries_and_symmetry():
    nx, ny, nz = 9, 6, 4
    cell = (3.90625, 3.90625, 5.0)
    prob = om.Problem(nx, ny, nz, *cell, Ms=1.0, A=0.0)
    octant = om.newell_octant(nx, ny, nz, *cell)
    full = om.newell_full(prob, octant)
    rng = np.random.default_rng(7)
    for _ in range(12):
        i, j, k = rng.integers(-(nx - 1), nx), rng.integers(-(ny - 1), ny), rng.integers(-(nz - 1), nz)
        N = om.newell_entry(i, j, k, *cell)
        got = full[:, k + nz - 1, j + ny - 1, i + nx - 1]
        assert np.allclose(got, N, rtol=1e-14, atol=1e-18)
    # N(-r) = N(r) as a tensor: diagonal even, off-diagonal odd in both of its axes
    assert np.allclose(full, full[:, ::-1, ::-1, ::-1], rtol=0, atol=1e-18)
    assert np.all(full[3:, nz - 1, ny - 1, nx - 1] == 0) or np.max(np.abs(full[3:, nz - 1, ny - 1, nx - 1])) < 1e-18
