"""Seeded synthetic inputs for the hysteresis workloads (shared by tests, bench and oracle checks).

This module only *generates* inputs: grids, material constants, initial
magnetisations and field sweeps.  It contains none of the method's
arithmetic, so the CUDA library and the CPU oracle can both be fed from it
without sharing any computation.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written out here so the same
seed gives the same bits on every machine and numpy version.

Workloads follow the thin-film geometry and material of muMAG Standard
Problem #1 as the paper gives them (Section 4: Ms = 8e5 A/m, A = 1.3e-11 J/m,
K = 500 J/m^3, easy axis along the long edge, field tilted 1 degree in plane,
1 mT field steps).  The paper's own runs used the SP1 film; only its geometry
and constants are used here, as synthetic stand-ins.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MU0 = 4e-7 * math.pi  # used only to express field values given in tesla as A/m

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of SplitMix64 started from ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.sqrt(np.sum(v * v, axis=0, keepdims=True))


def tilted_uniform_m(shape, seed: int, axis=(1.0, 0.0, 0.0), amplitude: float = 1e-3) -> np.ndarray:
    """Unit field (3, nz, ny, nx): normalize(axis + amplitude * xi), xi uniform in [-1,1]^3."""
    nz, ny, nx = shape
    xi = uniform(seed, 3 * nx * ny * nz, -1.0, 1.0).reshape(3, nz, ny, nx)
    v = np.asarray(axis, dtype=np.float64).reshape(3, 1, 1, 1) + amplitude * xi
    return np.ascontiguousarray(_unit(v))


def random_unit_m(shape, seed: int) -> np.ndarray:
    """Unit field (3, nz, ny, nx) with directions uniform on the sphere
    (z uniform in [-1,1], azimuth uniform)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    u = uniform(seed, 2 * n)
    z = 2.0 * u[:n] - 1.0
    phi = 2.0 * math.pi * u[n:]
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    m = np.stack([r * np.cos(phi), r * np.sin(phi), z]).reshape(3, nz, ny, nx)
    return np.ascontiguousarray(m)


def field_direction(tilt_deg: float = 1.0) -> np.ndarray:
    """In-plane unit vector tilted ``tilt_deg`` from +x toward +y."""
    t = math.radians(tilt_deg)
    return np.array([math.cos(t), math.sin(t), 0.0])


def sp1_sweep(max_mT: float = 50.0, step_mT: float = 1.0, tilt_deg: float = 1.0) -> np.ndarray:
    """Field values (n, 3) in A/m: descending +max..-max, then ascending
    -max+step..+max, along the tilted direction (201 values for 50 mT / 1 mT)."""
    n = int(round(max_mT / step_mT))
    desc = [max_mT - step_mT * i for i in range(2 * n + 1)]
    asc = [-max_mT + step_mT * i for i in range(1, 2 * n + 1)]
    b = np.array(desc + asc) * 1e-3  # tesla
    return np.outer(b / MU0, field_direction(tilt_deg))


@dataclasses.dataclass
class Workload:
    """One synthetic workload: grid, material and sweep (SI units)."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    Ms: float = 8.0e5
    A: float = 1.3e-11
    K: float = 500.0
    u: tuple = (1.0, 0.0, 0.0)
    tol: float = 1e-5
    seed: int = 1405
    max_mT: float = 50.0
    step_mT: float = 1.0
    tilt_deg: float = 1.0
    K_cell: np.ndarray | None = None  # per-cell K (nz, ny, nx) or None
    u_cell: np.ndarray | None = None  # per-cell easy axes (3, nz, ny, nx) or None
    H_list: np.ndarray | None = None  # explicit field values (n, 3) A/m, else the SP1 sweep

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def ncells(self):
        return self.nx * self.ny * self.nz

    def initial_m(self) -> np.ndarray:
        return tilted_uniform_m(self.shape, self.seed)

    def fields(self) -> np.ndarray:
        if self.H_list is not None:
            return self.H_list
        return sp1_sweep(self.max_mT, self.step_mT, self.tilt_deg)


def film_32x16x1() -> Workload:
    """1000 x 500 x 20 nm film on 32 x 16 x 1 cells (31.25 x 31.25 x 20 nm)."""
    return Workload("film_32x16x1", 32, 16, 1, 31.25e-9, 31.25e-9, 20e-9)


def film_512x256x4() -> Workload:
    """2000 x 1000 x 20 nm film on 512 x 256 x 4 cells (3.90625 x 3.90625 x 5 nm);
    padded FFT grid 1024 x 512 x 8."""
    return Workload("film_512x256x4", 512, 256, 4, 2000e-9 / 512, 1000e-9 / 256, 5e-9)


def film_128x64x2() -> Workload:
    """500 x 250 x 10 nm film on 128 x 64 x 2 cells (3.90625 x 3.90625 x 5 nm) with the
    uniform material of the 512 x 256 x 4 film: a quarter-size loop at the same cell size."""
    return Workload("film_128x64x2", 128, 64, 2, 500e-9 / 128, 250e-9 / 64, 5e-9)


def film_128x64x2_random_K() -> Workload:
    """500 x 250 x 10 nm film on 128 x 64 x 2 cells, per-cell K uniform in [300, 700] J/m^3."""
    w = Workload("film_128x64x2_randK", 128, 64, 2, 500e-9 / 128, 250e-9 / 64, 5e-9)
    w.K_cell = uniform(w.seed, w.ncells, 300.0, 700.0).reshape(w.shape)
    return w


def voronoi_grains(shape, cell, count: int, seed: int) -> np.ndarray:
    """Grain index (nz, ny, nx) of every cell: ``count`` seed points uniform in
    the box, each cell (by its centre) to the nearest seed in Euclidean
    distance, ties to the lower seed index."""
    nz, ny, nx = shape
    dx, dy, dz = cell
    pts = uniform(seed, 3 * count).reshape(count, 3) * np.array([nx * dx, ny * dy, nz * dz])
    xs = (np.arange(nx) + 0.5) * dx
    ys = (np.arange(ny) + 0.5) * dy
    grain = np.empty(shape, dtype=np.int32)
    dxy = (xs[None, None, :] - pts[:, 0, None, None]) ** 2 + (ys[None, :, None] - pts[:, 1, None, None]) ** 2
    for z in range(nz):
        d = dxy + ((z + 0.5) * dz - pts[:, 2, None, None]) ** 2
        grain[z] = np.argmin(d, axis=0)  # first minimum: ties go to the lower index
    return grain


def ramp_sweep(max_T: float, step_T: float, axis=(1.0, 0.0, 0.0)) -> np.ndarray:
    """Field values (n, 3) in A/m along ``axis``: 0 -> +max_T in step_T steps,
    then down to -max_T (481 values for 8 T / 50 mT)."""
    n = int(round(max_T / step_T))
    b = [step_T * i for i in range(n + 1)] + [max_T - step_T * i for i in range(1, 2 * n + 1)]
    return np.outer(np.array(b) / MU0, np.asarray(axis, dtype=np.float64))


def granular_cube(n: int = 256, grains: int = 64, seed: int = 1405, edge: float = 512e-9) -> Workload:
    """Granular hard-magnet cube: ``edge`` per side on n^3 cubic cells,
    ``grains`` Voronoi grains from seeded points, each grain with its own
    uniaxial easy axis uniform on the sphere; K = 4.3e6 J/m^3,
    Ms = 1.28e6 A/m, A = 7.7e-12 J/m; initial m = +x with the seeded 1e-3
    tilt; field along x, 0 -> +8 T -> -8 T in 50 mT steps."""
    h = edge / n
    w = Workload(f"cube_{n}^3_{grains}grains", n, n, n, h, h, h, Ms=1.28e6, A=7.7e-12, K=4.3e6, seed=seed)
    grain = voronoi_grains(w.shape, (h, h, h), grains, seed)
    axes = random_unit_m((1, 1, grains), seed + 1).reshape(3, grains)
    w.u_cell = np.ascontiguousarray(axes[:, grain])
    w.H_list = ramp_sweep(8.0, 0.05)
    return w


def batch_films(count: int = 64, seed: int = 1405, max_mT: float = 50.0, step_mT: float = 2.0):
    """``count`` films of uneven size on 3.90625 nm cubic cells: nx uniform in
    64..512, aspect a uniform in [1, 4], ny = clamp(round(nx / a), 32, 256),
    nz uniform in 1..4, K uniform in [0, 2000] J/m^3 (the 32x16x1 material
    otherwise), each with its own +-max_mT sweep in step_mT steps."""
    u = uniform(seed, 4 * count).reshape(count, 4)
    films = []
    for i in range(count):
        nx = 64 + int(u[i, 0] * 449)
        a = 1.0 + 3.0 * u[i, 1]
        ny = int(min(256, max(32, round(nx / a))))
        nz = 1 + int(u[i, 2] * 4)
        h = 3.90625e-9
        w = Workload(f"film{i}_{nx}x{ny}x{nz}", nx, ny, nz, h, h, h, K=2000.0 * float(u[i, 3]),
                     seed=seed + i, max_mT=max_mT, step_mT=step_mT)
        films.append(w)
    return films


WORKLOADS = {
    "film_32x16x1": film_32x16x1,
    "film_512x256x4": film_512x256x4,
    "film_128x64x2_randK": film_128x64x2_random_K,
    "film_128x64x2": film_128x64x2,
}

# bulk workloads (a different material and field protocol)
BULK_WORKLOADS = {
    "cube_256": granular_cube,
    # the same 512^3 padded grid with fewer cells (~2 GB on the device): the
    # case the bulk kernels are profiled on
    "cube_160": lambda: granular_cube(160, 64, edge=320e-9),
    # the same recipe (2 nm cells, 64 grains, 481-value ramp) on 64^3 cells:
    # small enough for whole FP32 and FP64 loops to be compared
    "cube_64": lambda: granular_cube(64, 64, edge=128e-9),
}
