"""Fixed values from the paper and from closed forms (tests/golden)."""
import json
import math
import os

import numpy as np

from paper_1405_2728_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_workloads_use_the_papers_sp1_material():
    g = json.load(open(os.path.join(GOLDEN, "sp1_material.json")))
    for make in inputs.WORKLOADS.values():
        w = make()
        assert (w.Ms, w.A) == (g["Ms_A_per_m"], g["A_J_per_m"])
        assert w.tilt_deg == g["tilt_deg"] and w.max_mT == g["field_max_mT"] and w.step_mT == g["field_step_mT"]
    assert inputs.film_512x256x4().K == g["K_J_per_m3"]


def test_sweep_values_and_tilt():
    H = inputs.sp1_sweep()
    assert H.shape == (201, 3)
    b = H @ inputs.field_direction(1.0) * inputs.MU0 * 1e3  # mT along the tilted axis
    assert np.allclose(b[:101], np.arange(50, -51, -1), atol=1e-9)
    assert np.allclose(b[101:], np.arange(-49, 51, 1), atol=1e-9)
    assert abs(math.degrees(math.atan2(H[0, 1], H[0, 0])) - 1.0) < 1e-12


def test_stoner_wohlfarth_table_matches_closed_form():
    for line in open(os.path.join(GOLDEN, "stoner_wohlfarth.txt")):
        if line.startswith("#") or not line.strip():
            continue
        psi, h = map(float, line.split())
        p = math.radians(psi)
        assert abs((math.cos(p) ** (2 / 3) + math.sin(p) ** (2 / 3)) ** -1.5 - h) < 6e-6


def test_splitmix64_known_sequence():
    # SplitMix64 reference outputs for seed 0 (first three values of the published generator)
    z = inputs.splitmix64(0, 3)
    assert [hex(int(v)) for v in z] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]
    u = inputs.uniform(1405, 1000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.05


def test_granular_cube_inputs():
    # small instance of the granular-cube generator: Voronoi grains by brute
    # force, unit axes, the 0 -> +8 T -> -8 T ramp in 50 mT steps
    w = inputs.granular_cube(10, 5, seed=7, edge=20e-9)
    assert (w.Ms, w.A, w.K) == (1.28e6, 7.7e-12, 4.3e6)
    assert w.u_cell.shape == (3, 10, 10, 10)
    assert np.allclose(np.linalg.norm(w.u_cell, axis=0), 1.0, atol=1e-14)
    pts = inputs.uniform(7, 15).reshape(5, 3) * 20e-9
    grain = inputs.voronoi_grains((10, 10, 10), (2e-9,) * 3, 5, 7)
    for (z, y, x) in [(0, 0, 0), (9, 9, 9), (3, 7, 1), (5, 0, 8)]:
        c = (np.array([x, y, z]) + 0.5) * 2e-9
        d = np.sum((pts - c) ** 2, axis=1)
        assert grain[z, y, x] == int(np.argmin(d))
    # each grain's cells share one axis
    for gi in range(5):
        sel = grain == gi
        if sel.any():
            ax = w.u_cell[:, sel]
            assert np.allclose(ax, ax[:, :1])
    H = inputs.ramp_sweep(8.0, 0.05)
    assert H.shape == (481, 3)
    b = H[:, 0] * inputs.MU0
    assert abs(b[0]) < 1e-15 and abs(b[160] - 8.0) < 1e-12 and abs(b[-1] + 8.0) < 1e-12
    assert np.all(np.diff(b[:161]) > 0) and np.all(np.diff(b[160:]) < 0)
    assert np.all(H[:, 1:] == 0)


def test_study_directions_and_sweep():
    # SP1 field directions (1 degree off each edge) and the +50 -> -50 -> +50 mT sweep
    from paper_1405_2728_gb300 import study
    h = study.direction("short")
    assert abs(np.linalg.norm(h) - 1) < 1e-15 and abs(math.degrees(math.atan2(h[0], h[1])) - 1.0) < 1e-12
    h = study.direction("long")
    assert abs(math.degrees(math.atan2(h[1], h[0])) - 1.0) < 1e-12
    H = study.sweep_fields(h, 50.0, 0.5)
    assert H.shape == (401, 3)
    b = H @ h * inputs.MU0 * 1e3
    assert abs(b[0] - 50) < 1e-9 and abs(b[200] + 50) < 1e-9 and abs(b[-1] - 50) < 1e-9
    # loop metrics of a hand-made loop: <m>.h = tanh((H - Hc) / w) on the way down
    hh = b * 1e-3 / inputs.MU0
    p = np.tanh((b + 7.25) / 2.0)
    mavg = np.outer(p, h)
    met = study.loop_metrics(H, mavg, h)
    assert met["H_sw"] * inputs.MU0 * 1e3 == -7.5
    assert -7.5 < met["H_c"] * inputs.MU0 * 1e3 < -7.0
    assert abs(met["M_r"][0] - np.tanh(7.25 / 2.0) * h[0]) < 1e-12


def test_batch_films_ranges_and_determinism():
    films = inputs.batch_films(64)
    assert len(films) == 64
    for w in films:
        assert 64 <= w.nx <= 512 and 32 <= w.ny <= 256 and 1 <= w.nz <= 4
        assert w.dx == w.dy == w.dz == 3.90625e-9 and 0.0 <= w.K < 2000.0
        assert (w.max_mT, w.step_mT) == (50.0, 2.0) and w.fields().shape == (101, 3)
    again = inputs.batch_films(64)
    assert [(w.nx, w.ny, w.nz, w.K) for w in films] == [(w.nx, w.ny, w.nz, w.K) for w in again]
    assert len({(w.nx, w.ny, w.nz) for w in films}) > 32  # uneven sizes


def test_bench_algorithmic_model_film():
    # pass-model bytes per kernel at 512x256x4 (F = 3 N s, W = 3 (Px/2+1) ny nz 2 s,
    # T = 6 (Px/2+1) max(1, Pz/2) (Py/2+1) s)
    import bench
    nx, ny, nz, Px, Py, Pz = 512, 256, 4, 1024, 512, 8
    for s in (8, 4):
        F = 3 * nx * ny * nz * s
        W = 3 * (Px // 2 + 1) * ny * nz * 2 * s
        T = 6 * (Px // 2 + 1) * (Pz // 2) * (Py // 2 + 1) * s
        info = {"nx": nx, "ny": ny, "nz": nz, "px": Px, "py": Py, "pz": Pz, "spectrum_bytes": W, "tensor_bytes": T,
                "bulk_layout": 0}
        mdl = bench.algorithmic_model(info, s)
        assert mdl["xfwd_step"]["bytes"] == 3 * F + W
        assert mdl["yz_conv"]["bytes"] == 2 * W + T
        assert mdl["xinv_local_bb"]["bytes"] == W + 4 * F
        if s == 8:  # 63 + 76 + 76 MB per iteration
            assert [round(mdl[k]["bytes"] / 1e6) for k in ("xfwd_step", "yz_conv", "xinv_local_bb")] == [63, 76, 76]
        assert all(v["flops"] > 0 for v in mdl.values())
    info["bulk_layout"] = 1
    mdl = bench.algorithmic_model(info, 4)
    assert set(mdl) == {"xfwd_step", "y_fwd", "z_conv", "y_inv", "xinv_local_bb"}
