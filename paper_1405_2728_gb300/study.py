"""Convergence study of the SP1 hysteresis loops (Section 4).

The paper reports three things about its Standard Problem #1 loops.  Refining
the cells from 10 nm to 5 nm leaves the loops unchanged.  Halving the field
step from 1 mT to 0.5 mT leaves them unchanged.  The remanent state is the
same whether the field runs along the long or the short edge.  This module
recomputes those loops with the library (FP64 or FP32) and reports, per
discretisation and field direction:

* the switching field H_sw: the first field on the descending branch where
  <m>.h < 0;
* the coercive field H_c: that zero crossing, linearly interpolated;
* the remanence M_r: <m> at zero field on the descending branch;
* the evaluation count and the wall time of the loop.

It also reports the remanent states of the two field directions against each
other (mean |m_long - m_short| over the cells).

Geometry and material are those of the SP1 film (inputs.py): 2000 x 1000 x
20 nm, long edge along x (the easy axis).  Field directions are 1 degree in
plane off the long edge (toward +y) and off the short edge (toward +x).  The
sweep is +50 -> -50 -> +50 mT.  The start is saturated along the field, with
the seeded 1e-3 tilt.

    python -m paper_1405_2728_gb300.study [--precision fp64|fp32|f32x2] [--cells 10,5] [--steps 1,0.5]
                                          [--tau-rule alternate|adaptive]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs, mm

EDGE = (2000e-9, 1000e-9, 20e-9)


def direction(edge: str, tilt_deg: float = 1.0) -> np.ndarray:
    """Unit field direction: 'long' = x tilted toward +y, 'short' = y tilted toward +x."""
    t = math.radians(tilt_deg)
    if edge == "long":
        return np.array([math.cos(t), math.sin(t), 0.0])
    return np.array([math.sin(t), math.cos(t), 0.0])


def sweep_fields(hhat: np.ndarray, max_mT: float = 50.0, step_mT: float = 1.0) -> np.ndarray:
    """+max -> -max -> +max in step_mT along hhat, in A/m (n, 3)."""
    n = int(round(max_mT / step_mT))
    b = [max_mT - step_mT * i for i in range(2 * n + 1)] + [-max_mT + step_mT * i for i in range(1, 2 * n + 1)]
    return np.outer(np.array(b) * 1e-3 / inputs.MU0, hhat)


def loop_metrics(H: np.ndarray, mavg: np.ndarray, hhat: np.ndarray) -> dict:
    """H_sw, H_c (A/m, signed along hhat) and M_r (<m> at zero field) of the
    descending branch (the values before the field turns)."""
    h = H @ hhat
    p = mavg @ hhat
    nd = 1
    while nd < len(h) and h[nd] < h[nd - 1]:
        nd += 1
    out = {"H_sw": None, "H_c": None, "M_r": None}
    for i in range(1, nd):
        if p[i] < 0:
            out["H_sw"] = float(h[i])
            out["H_c"] = float(h[i - 1] + (h[i] - h[i - 1]) * p[i - 1] / (p[i - 1] - p[i]))
            break
    for i in range(nd):
        if abs(h[i]) < 1e-9 * max(1.0, abs(h[0])):
            out["M_r"] = [float(x) for x in mavg[i]]
            break
    return out


def run_loop(cell_nm: float, step_mT: float, edge: str, precision: int, tol: float = 1e-5, seed: int = 1405,
             tau_rule: int = mm.MM_TAU_ALTERNATE):
    """One SP1 loop.  Returns (metrics, remanent m (3, nz, ny, nx) as numpy, evals, seconds)."""
    import torch

    h = cell_nm * 1e-9
    nx, ny, nz = (int(round(L / h)) for L in EDGE)
    grid = mm.make_grid(nx, ny, nz, EDGE[0] / nx, EDGE[1] / ny, EDGE[2] / nz)
    prob = mm.mm_setup_geometry(grid, mm.make_material(8.0e5, 1.3e-11, 500.0), precision)
    hhat = direction(edge)
    H = sweep_fields(hhat, 50.0, step_mT)
    dt = torch.float32 if precision == mm.MM_FP32 else torch.float64
    m0 = inputs.tilted_uniform_m((nz, ny, nx), seed, axis=tuple(hhat))
    m = torch.from_numpy(m0).to(device="cuda", dtype=dt).contiguous()
    opts = mm.make_opts(tol=tol, max_iter=200000, tau_rule=tau_rule)
    i0 = int(np.argmin(np.abs(H @ hhat)[: len(H) // 2 + 1]))  # zero field on the descending branch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mavg = np.full((len(H), 3), np.nan)
    st1, mavg, res1 = mm.mm_hysteresis_sweep(prob, m, H[: i0 + 1], opts=opts, mavg=mavg[: i0 + 1])
    rem = m.double().cpu().numpy()
    mavg_full = np.full((len(H), 3), np.nan)
    mavg_full[: i0 + 1] = mavg
    st2, mavg_full, res2 = mm.mm_hysteresis_sweep(prob, m, H, start=i0 + 1, opts=opts, mavg=mavg_full)
    torch.cuda.synchronize()
    dt_s = time.perf_counter() - t0
    evals = sum(r.heff_evals for r in res1) + sum(r.heff_evals for r in res2[i0 + 1:])
    met = loop_metrics(H, mavg_full, hhat)
    met["converged"] = bool(st1 == mm.MM_OK and st2 == mm.MM_OK)
    met["grid"] = [nx, ny, nz]
    prob.close()
    return met, rem, evals, dt_s


def convergence_study(precision: int = mm.MM_FP64, cells_nm=(10.0, 5.0), steps_mT=(1.0, 0.5),
                      tau_rule: int = mm.MM_TAU_ALTERNATE):
    rows = []
    remanence = {}
    for c in cells_nm:
        for s in steps_mT:
            for edge in ("long", "short"):
                met, rem, ev, sec = run_loop(c, s, edge, precision, tau_rule=tau_rule)
                rows.append({"cell_nm": c, "step_mT": s, "field_edge": edge, **met,
                             "evals": int(ev), "seconds": sec})
                remanence[(c, s, edge)] = rem
    # remanent states of the two field directions against each other
    rem_cmp = []
    for c in cells_nm:
        for s in steps_mT:
            a, b = remanence[(c, s, "long")], remanence[(c, s, "short")]
            rem_cmp.append({"cell_nm": c, "step_mT": s,
                            "mean_abs_diff": float(np.mean(np.linalg.norm(a - b, axis=0))),
                            "mean_dot": float(np.mean(np.sum(a * b, axis=0)))})
    return rows, rem_cmp


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "f32x2"])
    ap.add_argument("--tau-rule", default="alternate", choices=["alternate", "adaptive"],
                    help="step-size rule: alternate tau^1/tau^2 (Section 2) or the adaptive switch")
    ap.add_argument("--cells", default="10,5", help="cell sizes in nm, comma separated")
    ap.add_argument("--steps", default="1,0.5", help="field steps in mT, comma separated")
    args = ap.parse_args(argv)
    prec = {"fp64": mm.MM_FP64, "fp32": mm.MM_FP32, "f32x2": mm.MM_F32X2}[args.precision]
    rule = mm.MM_TAU_ADAPTIVE if args.tau_rule == "adaptive" else mm.MM_TAU_ALTERNATE
    rows, rem = convergence_study(prec, [float(x) for x in args.cells.split(",")],
                                  [float(x) for x in args.steps.split(",")], rule)
    mu0 = inputs.MU0
    for r in rows:  # fields in mT for reading
        for k in ("H_sw", "H_c"):
            if r[k] is not None:
                r[k + "_mT"] = r[k] * mu0 * 1e3
    print(json.dumps({"study": "sp1_convergence", "precision": args.precision, "tau_rule": args.tau_rule, "loops": rows,
                      "remanence_long_vs_short": rem}))


if __name__ == "__main__":
    main()
