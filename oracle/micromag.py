"""Float64 CPU oracle of the energy-minimising hysteresis method.

Test infrastructure only (tests, the smoke check and the benchmark's CPU
baseline); the product library never imports it.  Everything here is written
from the paper (Abert et al., "Efficient Energyminimization in
Finite-Difference Micromagnetics", arXiv 1405.2728) and from the textbook
definitions of the energy terms, as plainly as possible:

* effective field, Eq. (effective_field): H_eff = -(1/(mu0 Ms)) dU/dm.  On the
  grid this is taken cell-wise as H_i = -(1/(mu0 Ms V)) dU/dm_i, so that the
  discrete energy and field below are exactly consistent.
* demagnetisation, Section 3 ("FFT accelerated convolution" on a regular
  cuboid grid): H_d,i = -Ms sum_j N(r_i - r_j) m_j with the Newell tensor of
  ``newell_quad.c``; evaluated by a zero-padded FFT (scipy.fft as the library
  step) and, for the pins, by the direct O(N^2) sum.
* exchange (Section 4, A): six-neighbour finite differences with free faces,
  E_ex = A V sum_{neighbour pairs} |m_j - m_i|^2 / d^2.
* uniaxial anisotropy (Section 4, K, easy axis u): E_an = sum_i K_i V (1 - (m_i.u_i)^2).
* Zeeman: E_Z = -mu0 Ms V sum_i m_i . H_ext.
* minimiser, Section 2: projected direction g = m x (m x H) (Eq.
  projected_direction / the auxiliary fields of Eq. stepsize), the midpoint
  scheme Eq. (implicit_gradient_descent) solved in closed form, the two
  Barzilai-Borwein step sizes of Eq. (stepsize) used alternately, the first
  step from a small fixed guess, and the sup-norm stop rule.
* hysteresis driver, Section 4: one minimisation per field value, warm-started
  from the previous magnetisation.

Where the paper is silent or garbled, the readings taken are stated at the
function they affect: the descent sign of the step and the printed sign slip
of the projection (``projected_gradient``, ``cayley_step``), the alternation
order and the fallback for non-positive curvature (``bb_tau``), the first step
size tau0 = 1e-2/Ms and the stop quantity max|m x H|/Ms evaluated before
stepping (``minimize``), the restart of the step-size history at every field
value (``sweep``), the free exchange boundary (``exchange_field``) and
mu0 = 4 pi 1e-7 exactly (``MU0``).

Arrays: a vector field is float64 of shape (3, nz, ny, nx) (x fastest).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import scipy.fft

from . import build_oracle

MU0 = 4e-7 * np.pi  # vacuum permeability, exactly 4 pi 1e-7 (reading: pre-2019 SI value)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_oracle.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_newell_octant.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [dp]
        lib.oracle_newell_octant.restype = ctypes.c_int
        lib.oracle_newell_entry.argtypes = [ctypes.c_long] * 3 + [ctypes.c_double] * 3 + [dp]
        lib.oracle_newell_entry.restype = ctypes.c_int
        lib.oracle_newell_f.argtypes = [ctypes.c_double] * 3
        lib.oracle_newell_f.restype = ctypes.c_double
        lib.oracle_newell_g.argtypes = [ctypes.c_double] * 3
        lib.oracle_newell_g.restype = ctypes.c_double
        lib.oracle_quad_mant_dig.restype = ctypes.c_int
        _LIB = lib
    return _LIB


# ----------------------------------------------------------------------------
# Problem description
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Grid and material.  Lengths in m, Ms in A/m, A in J/m, K in J/m^3.

    K is a scalar or an array (nz, ny, nx); u is a unit 3-vector or an array
    (3, nz, ny, nx) of unit vectors (per-cell easy axes).
    """
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    Ms: float
    A: float
    K: object = 0.0
    u: object = (1.0, 0.0, 0.0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def V(self):
        return self.dx * self.dy * self.dz

    def K_cells(self):
        return np.broadcast_to(np.asarray(self.K, dtype=np.float64), self.shape)

    def u_cells(self):
        u = np.asarray(self.u, dtype=np.float64)
        if u.ndim == 1:
            u = u.reshape(3, 1, 1, 1)
        return np.broadcast_to(u, (3,) + self.shape)


# ----------------------------------------------------------------------------
# Newell tensor (quad precision, via newell_quad.c)
# ----------------------------------------------------------------------------

def newell_f(x, y, z):
    """Newell's f at one point (quad evaluation rounded to double)."""
    return _lib().oracle_newell_f(float(x), float(y), float(z))


def newell_g(x, y, z):
    """Newell's g at one point (quad evaluation rounded to double)."""
    return _lib().oracle_newell_g(float(x), float(y), float(z))


def newell_entry(i, j, k, dx, dy, dz):
    """All six components (xx, yy, zz, xy, xz, yz) at signed offset (i, j, k) cells."""
    out = (ctypes.c_double * 6)()
    if _lib().oracle_newell_entry(int(i), int(j), int(k), float(dx), float(dy), float(dz), out):
        raise ValueError("bad cell size")
    return np.array(out[:], dtype=np.float64)


def newell_octant(nx, ny, nz, dx, dy, dz):
    """Tensor on offsets 0<=i<nx, 0<=j<ny, 0<=k<nz: array (6, nz, ny, nx)."""
    out = np.empty((6, nz, ny, nx), dtype=np.float64)
    rc = _lib().oracle_newell_octant(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc:
        raise ValueError("oracle_newell_octant failed")
    return out


# Parity of each component under a sign flip of (x, y, z) offsets:
# diagonal entries are even in every coordinate, N_ab is odd in a and in b.
_ODD = {0: (0, 0, 0), 1: (0, 0, 0), 2: (0, 0, 0), 3: (1, 1, 0), 4: (1, 0, 1), 5: (0, 1, 1)}


def newell_full(prob_or_grid, octant=None):
    """Tensor on all offsets -(n-1)..(n-1): array (6, 2nz-1, 2ny-1, 2nx-1).

    Index [c, k + nz - 1, j + ny - 1, i + nx - 1] holds N_c at offset (i, j, k).
    """
    g = prob_or_grid
    nx, ny, nz = g.nx, g.ny, g.nz
    if octant is None:
        octant = newell_octant(nx, ny, nz, g.dx, g.dy, g.dz)
    ii = np.arange(-(nx - 1), nx)
    jj = np.arange(-(ny - 1), ny)
    kk = np.arange(-(nz - 1), nz)
    full = np.empty((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    for c in range(6):
        ox, oy, oz = _ODD[c]
        sx = np.where(ii < 0, -1.0, 1.0) if ox else np.ones_like(ii, dtype=float)
        sy = np.where(jj < 0, -1.0, 1.0) if oy else np.ones_like(jj, dtype=float)
        sz = np.where(kk < 0, -1.0, 1.0) if oz else np.ones_like(kk, dtype=float)
        block = octant[c][np.abs(kk)][:, np.abs(jj)][:, :, np.abs(ii)]
        full[c] = block * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    return full


def _sym(full):
    """3x3 index -> component of the 6-vector (xx, yy, zz, xy, xz, yz)."""
    return [[full[0], full[3], full[4]], [full[3], full[1], full[5]], [full[4], full[5], full[2]]]


# ----------------------------------------------------------------------------
# Field terms
# ----------------------------------------------------------------------------

class Demag:
    """Demagnetisation field by zero-padded FFT convolution (Section 3).

    Padding: 2n per axis (any P >= 2n - 1 gives the exact linear convolution);
    the tensor at offset d is placed at index d mod P, unused indices are 0.
    """

    def __init__(self, prob: Problem, full=None, workers=None):
        self.prob = prob
        self.workers = workers if workers is not None else (os.cpu_count() or 1)
        nx, ny, nz = prob.nx, prob.ny, prob.nz
        self.P = (2 * nz, 2 * ny, 2 * nx)
        if full is None:
            full = newell_full(prob)
        self.full = full
        padded = np.zeros((6,) + self.P)
        kk = np.arange(-(nz - 1), nz) % self.P[0]
        jj = np.arange(-(ny - 1), ny) % self.P[1]
        ii = np.arange(-(nx - 1), nx) % self.P[2]
        padded[:, kk[:, None, None], jj[None, :, None], ii[None, None, :]] = full
        self.Nhat = scipy.fft.rfftn(padded, axes=(1, 2, 3), workers=self.workers)

    def field(self, m):
        p = self.prob
        mp = np.zeros((3,) + self.P)
        mp[:, :p.nz, :p.ny, :p.nx] = m
        mh = scipy.fft.rfftn(mp, axes=(1, 2, 3), workers=self.workers)
        N = _sym(self.Nhat)
        Hh = np.empty_like(mh)
        for a in range(3):
            Hh[a] = -p.Ms * (N[a][0] * mh[0] + N[a][1] * mh[1] + N[a][2] * mh[2])
        H = scipy.fft.irfftn(Hh, s=self.P, axes=(1, 2, 3), workers=self.workers)
        return np.ascontiguousarray(H[:, :p.nz, :p.ny, :p.nx])


def demag_direct(prob: Problem, m, full=None, cells=None):
    """Direct sum H_d,i = -Ms sum_j N(r_i - r_j) m_j (no FFT), at all cells or
    at the listed flat cell indices.  Returns (3, ncells) for ``cells`` else (3, nz, ny, nx)."""
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    if full is None:
        full = newell_full(prob)
    N = _sym(full)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    targets = np.arange(nx * ny * nz) if cells is None else np.asarray(cells)
    out = np.empty((3, len(targets)))
    for t, flat in enumerate(targets):
        k, j, i = np.unravel_index(flat, (nz, ny, nx))
        dk = k - K + nz - 1
        dj = j - J + ny - 1
        di = i - I + nx - 1
        for a in range(3):
            out[a, t] = -prob.Ms * sum(np.sum(N[a][b][dk, dj, di] * m[b]) for b in range(3))
    if cells is None:
        return out.reshape((3, nz, ny, nx))
    return out


def exchange_field(prob: Problem, m):
    """H_ex,i = (2A/(mu0 Ms)) sum_{j in nb(i)} (m_j - m_i)/d^2; missing neighbours
    at the faces are absent (free boundary)."""
    H = np.zeros_like(m)
    c = 2.0 * prob.A / (MU0 * prob.Ms)
    for axis, d in ((3, prob.dx), (2, prob.dy), (1, prob.dz)):
        n = m.shape[axis]
        if n < 2:
            continue
        diff = np.diff(m, axis=axis) / (d * d)  # m_{i+1} - m_i on each pair
        lo = [slice(None)] * 4
        hi = [slice(None)] * 4
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        H[tuple(lo)] += c * diff
        H[tuple(hi)] -= c * diff
    return H


def anisotropy_field(prob: Problem, m):
    """H_an,i = (2 K_i/(mu0 Ms)) (m_i . u_i) u_i."""
    u = prob.u_cells()
    K = prob.K_cells()
    mu = np.sum(m * u, axis=0)
    return (2.0 * K * mu / (MU0 * prob.Ms))[None] * u


def heff(prob: Problem, m, Hext, demag: Demag):
    """Total effective field (A/m): demag + exchange + anisotropy + Zeeman."""
    H = demag.field(m) + exchange_field(prob, m) + anisotropy_field(prob, m)
    H += np.asarray(Hext, dtype=np.float64).reshape(3, 1, 1, 1)
    return H


def energy(prob: Problem, m, Hext, demag: Demag):
    """Energy terms in J: demag, exchange, anisotropy, Zeeman, total.

    E_d = -(mu0 Ms V/2) sum m.H_d (= (mu0 Ms^2 V/2) sum_ij m_i.N_ij m_j);
    E_ex over neighbour pairs; E_an = sum K V (1 - (m.u)^2); E_Z = -mu0 Ms V sum m.H_ext.
    """
    V, Ms = prob.V, prob.Ms
    Ed = -0.5 * MU0 * Ms * V * float(np.sum(m * demag.field(m)))
    Eex = 0.0
    for axis, d in ((3, prob.dx), (2, prob.dy), (1, prob.dz)):
        if m.shape[axis] > 1:
            Eex += prob.A * V * float(np.sum(np.diff(m, axis=axis) ** 2)) / (d * d)
    u = prob.u_cells()
    Ean = float(np.sum(prob.K_cells() * V * (1.0 - np.sum(m * u, axis=0) ** 2)))
    EZ = -MU0 * Ms * V * float(np.sum(m * np.asarray(Hext, dtype=np.float64).reshape(3, 1, 1, 1)))
    return {"demag": Ed, "exchange": Eex, "anisotropy": Ean, "zeeman": EZ,
            "total": Ed + Eex + Ean + EZ}


# ----------------------------------------------------------------------------
# Minimiser (Section 2)
# ----------------------------------------------------------------------------

def projected_gradient(m, H):
    """g = m x (m x H): the auxiliary field g_k of Eq. (stepsize).

    Equals (m.H) m - H = -(tangential part of H), i.e. (mu0 Ms V) times the
    tangent-plane projection of dU/dm (the printed second line of
    Eq. projected_direction carries a sign slip; the projection itself is
    v - (v.m) m)."""
    return np.cross(m, np.cross(m, H, axis=0), axis=0)


def max_torque(m, H, Ms):
    """Stop quantity max_i |m_i x H_i| / Ms (reading of the sup-norm rule)."""
    return float(np.max(np.linalg.norm(np.cross(m, H, axis=0), axis=0))) / Ms


def cayley_step(m, g, tau):
    """Closed-form solution of the midpoint scheme, Eq. (implicit_gradient_descent),
    in its descent orientation m' = m + tau ((m + m')/2) x (m x H) with the
    printed tau replaced by -tau (tau > 0 from Eq. stepsize):

        m' = [(1 - tau^2 |g|^2/4) m - tau g] / (1 + tau^2 |g|^2/4),

    valid for |m| = 1 and g = m x (m x H) (so g is tangent to m)."""
    q = 0.25 * tau * tau * np.sum(g * g, axis=0)
    return ((1.0 - q) * m - tau * g) / (1.0 + q)


def normalize_step(m, g, tau):
    """Variant: explicit projected step Eq. (projected_gradient_descent) in
    descent orientation, followed by renormalisation: m' = (m - tau g)/|m - tau g|."""
    v = m - tau * g
    return v / np.linalg.norm(v, axis=0)


def bb_tau(k, s, y, tau0, rule="alternate", kappa=0.5):
    """Step size of Eq. (stepsize): tau^1 = sum s.s / sum s.y on odd k,
    tau^2 = sum s.y / sum y.y on even k (alternating, Section 2).

    rule="adaptive": the paper names a "more elaborate switch" between the
    two sizes without giving it.  Reading: the adaptive Barzilai-Borwein rule
    of Zhou, Gao and Dai (Comput. Optim. Appl. 35 (2006) 69): take the short
    size tau^2 when tau^2 / tau^1 = (s.y)^2 / ((s.s)(y.y)) < kappa, else the
    long size tau^1, at every k >= 1.  The ratio is the squared cosine of
    the angle between s and y; a small value means the last step met strongly
    varying curvature, where the short size is the safer one.

    The paper is silent on non-positive curvature (sum s.y <= 0) and zero
    denominators.  Reading: use sqrt(sum s.s / sum y.y) (= |s|/|y|, the
    magnitude both quotients share when s and y are parallel) if that is
    finite and positive, else tau0.  A fixed tau0 fallback crawls through
    negative-curvature regions at tau0-sized steps and fails to converge
    near switching fields."""
    ss = np.float64(np.sum(s * s))
    sy = np.float64(np.sum(s * y))
    yy = np.float64(np.sum(y * y))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        if rule == "adaptive":
            tau = sy / yy if (sy * sy) < kappa * (ss * yy) else ss / sy
        else:
            tau = ss / sy if (k % 2 == 1) else sy / yy
        if not (np.isfinite(tau) and tau > 0):
            tau = np.sqrt(ss / yy)
    if not (np.isfinite(tau) and tau > 0):
        tau = tau0
    return float(tau)


@dataclasses.dataclass
class MinResult:
    m: np.ndarray
    iters: int          # number of steps taken
    heff_evals: int     # effective-field evaluations (iters + 1)
    max_torque: float   # final max |m x H| / Ms
    converged: bool
    taus: list


def minimize(prob: Problem, m0, Hext, demag: Demag, tol=1e-5, tau0=None, max_iter=100000,
             step="cayley", record_taus=False, tau_rule="alternate", kappa=0.5):
    """Projected Barzilai-Borwein minimisation at one field value (Section 2).

    k counts steps within this minimisation.  Each pass: H = H_eff(m_k),
    g_k = m_k x (m_k x H); stop if max|m_k x H|/Ms < tol; stop unconverged
    after max_iter steps; tau_k = tau0 for k = 0 else the BB value (``bb_tau``
    with ``tau_rule``); step.
    """
    Ms = prob.Ms
    if tau0 is None:
        tau0 = 1e-2 / Ms
    stepf = cayley_step if step == "cayley" else normalize_step
    m = np.array(m0, dtype=np.float64, copy=True)
    m_prev = g_prev = None
    k = 0
    evals = 0
    taus = []
    while True:
        H = heff(prob, m, Hext, demag)
        g = projected_gradient(m, H)
        evals += 1
        t = max_torque(m, H, Ms)
        if t < tol:
            return MinResult(m, k, evals, t, True, taus)
        if k >= max_iter:
            return MinResult(m, k, evals, t, False, taus)
        tau = tau0 if k == 0 else bb_tau(k, m - m_prev, g - g_prev, tau0, tau_rule, kappa)
        if record_taus:
            taus.append(tau)
        m_prev, g_prev = m, g
        m = stepf(m, g, tau)
        k += 1


def sweep(prob: Problem, m0, H_list, demag: Demag, tol=1e-5, tau0=None, max_iter=100000,
          step="cayley", tau_rule="alternate", kappa=0.5):
    """Hysteresis driver (Section 4): minimise once per field value, starting
    from the previous magnetisation; the BB history restarts at every field
    value.  Returns (mavg (n,3), list of MinResult without m, final m)."""
    m = np.array(m0, dtype=np.float64, copy=True)
    mavg = np.empty((len(H_list), 3))
    results = []
    for n, H in enumerate(H_list):
        r = minimize(prob, m, H, demag, tol=tol, tau0=tau0, max_iter=max_iter, step=step,
                     tau_rule=tau_rule, kappa=kappa)
        m = r.m
        mavg[n] = m.reshape(3, -1).mean(axis=1)
        results.append(dataclasses.replace(r, m=None))
    return mavg, results, m


def loop_metrics(H_list, mavg):
    """Switching field, coercive field and remanence of a loop whose first
    branch descends.  hhat = direction of the first field value.

    H_sw: first field on the descending branch where <m>.hhat < 0.
    H_c : zero crossing of <m>.hhat on that branch, linearly interpolated.
    M_r : <m_x> at zero field on the descending branch (nan if absent).
    Fields are returned as signed magnitudes along hhat (A/m)."""
    H_list = np.asarray(H_list, dtype=np.float64)
    hhat = H_list[0] / np.linalg.norm(H_list[0])
    h = H_list @ hhat
    p = mavg @ hhat
    n_desc = 1
    while n_desc < len(h) and h[n_desc] < h[n_desc - 1]:
        n_desc += 1
    H_sw = H_c = np.nan
    for n in range(1, n_desc):
        if p[n] < 0:
            H_sw = h[n]
            H_c = h[n - 1] + (h[n] - h[n - 1]) * p[n - 1] / (p[n - 1] - p[n])
            break
    M_r = np.nan
    for n in range(n_desc):
        if abs(h[n]) < 1e-9 * max(1.0, abs(h[0])):
            M_r = mavg[n, 0]
            break
    return {"H_sw": H_sw, "H_c": H_c, "M_r": M_r}


# ----------------------------------------------------------------------------
# Implicit adjoint at a converged minimum (differentiation extension; not in
# the paper).  At a minimum the torque vanishes, P_m H(m; K) = 0 with
# P_m w = w - (m.w) m.  Linearising gives A dm = P_m(dH/dK) dK with the
# tangent-plane operator A v = (m.H) v - P_m(L v), L v = H_eff(v) without the
# external field (all other terms are linear in m).  For an objective J(m),
# dJ/dK_i = lambda . P_m(dH/dK_i) with A lambda = P_m(dJ/dm).
# ----------------------------------------------------------------------------

def project(m, w):
    """Tangent-plane projection w - (m.w) m, per cell."""
    return w - np.sum(m * w, axis=0)[None] * m


def hessian_vec(prob: Problem, m, H, v, demag: Demag):
    """A v = P_m((m.H) v - L v), i.e. (m.H) v - P_m(L v) for a tangent field v;
    H = H_eff(m).  Projecting the whole product keeps iterates tangent: a
    normal component left by rounding would otherwise be multiplied by m.H
    (large and negative near the film's ends) at every product."""
    Lv = heff(prob, v, (0.0, 0.0, 0.0), demag)
    return project(m, np.sum(m * H, axis=0)[None] * v - Lv)


def adjoint_solve(prob: Problem, m, Hext, rhs, demag: Demag, tol=1e-12, max_iter=10000):
    """Conjugate gradients for A lam = P_m(rhs) on tangent fields."""
    H = heff(prob, m, Hext, demag)
    b = project(m, rhs)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    bb = rr
    it = 0
    while rr > tol * tol * bb and it < max_iter:
        Ap = hessian_vec(prob, m, H, p, demag)
        alpha = rr / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def dJ_dK(prob: Problem, m, Hext, dJdm, demag: Demag, tol=1e-12):
    """Gradient of an objective J(m*(K)) with respect to the per-cell K at a
    converged minimum m*: lam . P_m(dH/dK_i), dH_i/dK_i = (2/(mu0 Ms)) (m_i.u_i) u_i."""
    lam, it = adjoint_solve(prob, m, Hext, dJdm, demag, tol=tol)
    u = prob.u_cells()
    mu = np.sum(m * u, axis=0)
    dH = (2.0 / (MU0 * prob.Ms)) * mu[None] * u
    return np.sum(lam * project(m, dH), axis=0), it
