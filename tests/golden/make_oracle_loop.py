"""Write the oracle's descending branch of a film's hysteresis loop.

Calls only the CPU oracle (``oracle/``) and the seeded input generators.  The
default workload is the thin film of Section 4 (2000 x 1000 x 20 nm on
512 x 256 x 4 cells, Ms = 8e5 A/m, A = 1.3e-11 J/m, K = 500 J/m^3 along x,
field 1 degree off x in 1 mT steps, stop at max|m x H|/Ms < 1e-5);
``--workload film_128x64x2`` takes the same material on a 500 x 250 x 10 nm
film with the same cells, whose whole branch the oracle finishes in about an
hour on a few host cores.  The sweep starts at
+50 mT from the seeded tilted state and runs down the descending branch one
field value at a time, warm-started from the previous magnetisation, until
the first value past 0 mT whose mean magnetisation points against the field
(the switching field).  That covers the remanence (0 mT) and the switching
field, the two loop results compared against the CUDA library.

Output (``<workload>_descending.json``): the input hash, and per field
value the field (A/m), <m>, the evaluation count, the final torque and the
convergence flag.  A state file given by ``--state`` lets a long run resume;
it holds the current magnetisation and is not part of the stored values.

Usage:  python tests/golden/make_oracle_loop.py [--workload NAME] [--state PATH] [--workers N]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import micromag as om  # noqa: E402
from paper_1405_2728_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def input_hash(w, m0, H_list) -> str:
    """SHA-256 over the grid, material, tolerance, start state and field list."""
    h = hashlib.sha256()
    h.update(json.dumps([w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.Ms, w.A, w.K, list(w.u), w.tol]).encode())
    h.update(np.ascontiguousarray(m0, dtype=np.float64).tobytes())
    h.update(np.ascontiguousarray(H_list, dtype=np.float64).tobytes())
    return h.hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--state", default=None, help="resume file (npz) for the current magnetisation")
    ap.add_argument("--workers", type=int, default=None, help="FFT threads of the oracle")
    ap.add_argument("--max-iter", type=int, default=100000)
    ap.add_argument("--workload", default="film_512x256x4", choices=["film_512x256x4", "film_128x64x2"])
    ap.add_argument("--whole-loop", action="store_true",
                    help="all 201 field values (descending and ascending branch), not just past the switch")
    args = ap.parse_args()

    w = inputs.WORKLOADS[args.workload]()
    OUT = os.path.join(HERE, f"{w.name}_{'loop' if args.whole_loop else 'descending'}.json")
    prob = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K, u=w.u)
    H_all = w.fields()
    n_desc = len(H_all) if args.whole_loop else 101  # +50 ... -50 mT (and back)
    H_desc = H_all[:n_desc]
    m0 = w.initial_m()
    key = input_hash(w, m0, H_all)
    hhat = inputs.field_direction(w.tilt_deg)

    rec = {"workload": w.name, "input_hash": key, "tol": w.tol, "max_iter": args.max_iter,
           "field_mT": [], "H": [], "mavg": [], "heff_evals": [], "max_torque": [], "converged": [],
           "seconds": [], "complete": False}
    m = m0
    if args.state and os.path.exists(args.state) and os.path.exists(OUT):
        prev = json.load(open(OUT))
        st = np.load(args.state)
        if prev.get("input_hash") == key and int(st["count"]) == len(prev["mavg"]):
            rec = prev
            m = st["m"]
            print(f"resuming after {len(rec['mavg'])} field values", flush=True)

    demag = om.Demag(prob, workers=args.workers)
    for n in range(len(rec["mavg"]), n_desc):
        if rec["complete"]:
            break
        t0 = time.time()
        r = om.minimize(prob, m, H_desc[n], demag, tol=w.tol, max_iter=args.max_iter)
        m = r.m
        mavg = m.reshape(3, -1).mean(axis=1)
        b_mT = float(H_desc[n] @ hhat) * om.MU0 * 1e3
        rec["field_mT"].append(round(b_mT, 9))
        rec["H"].append([float(v) for v in H_desc[n]])
        rec["mavg"].append([float(v) for v in mavg])
        rec["heff_evals"].append(int(r.heff_evals))
        rec["max_torque"].append(float(r.max_torque))
        rec["converged"].append(bool(r.converged))
        rec["seconds"].append(round(time.time() - t0, 3))
        if args.whole_loop:
            rec["complete"] = n + 1 == n_desc
        elif b_mT < 0 and float(mavg @ hhat) < 0:
            rec["complete"] = True
        tmp = OUT + ".tmp"
        with open(tmp, "w") as f:
            json.dump(rec, f, indent=1)
        if args.state:
            np.savez(args.state + ".tmp.npz", m=m, count=len(rec["mavg"]))
            os.replace(args.state + ".tmp.npz", args.state)
        os.replace(tmp, OUT)
        print(f"{b_mT:+7.2f} mT  <m>=({mavg[0]:+.6f},{mavg[1]:+.6f},{mavg[2]:+.6f})  "
              f"evals {r.heff_evals:6d}  conv {r.converged}  {time.time() - t0:8.1f} s", flush=True)


if __name__ == "__main__":
    main()
