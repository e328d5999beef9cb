"""Helpers shared by the GPU parity tests: the same seeded problem on the
CUDA library (through the C ABI) and on the CPU oracle."""
import numpy as np
import torch

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_pair(mm, nx, ny, nz, cell, Ms=8e5, A=1.3e-11, K=500.0, u=(1.0, 0.0, 0.0), K_cell=None, u_cell=None,
              precision=0):
    grid = mm.make_grid(nx, ny, nz, *cell)
    mat = mm.make_material(Ms, A, K, u, K_cell=K_cell, u_cell=u_cell)
    prob = mm.mm_setup_geometry(grid, mat, precision)
    oprob = om.Problem(nx, ny, nz, *cell, Ms=Ms, A=A, K=K if K_cell is None else K_cell,
                       u=u if u_cell is None else u_cell)
    return prob, oprob


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)
