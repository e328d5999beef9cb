"""Loop parity against the CPU oracle's stored hysteresis loops (Section 4):
the GPU sweeps the same seeded film over the same field values and its loop
is compared with the oracle's, stored in tests/golden/ by the committed
script beside it (make_oracle_loop.py, which calls only the oracle).

* film_128x64x2_loop.json: the whole 201-value loop (+50 -> -50 -> +50 mT) of
  a 500 x 250 x 10 nm film on the headline cell size;
* film_128x64x2_descending.json: its descending branch;
* film_512x256x4_descending.json: the headline film's descending branch, as far
  as the oracle has got on the host (the stored prefix is compared).

The energy is non-convex, so near a switching field rounding may pick a
different branch (the loops are compared, not the states one by one there):
the switching field of each branch -- the first field value past zero where
<m>.h changes sign -- must agree within one field step, the remanence <m_x>
at 0 mT on the descending branch within 1e-3, and <m> per field value within
1e-3 while neither loop has switched."""
import importlib.util
import json
import os

import numpy as np
import pytest
import torch

from paper_1405_2728_gb300 import inputs
from gpu_cases import dev

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# FP32 is compared on the 128 x 64 x 2 loops; on the 512 x 256 x 4 film its
# float rounding stalls the step-size sums near the tolerance, and some field
# values need more than the stored run's 1e5-iteration cap
CASES = [(f, wl, p) for f, wl, precs in (("film_128x64x2_loop.json", "film_128x64x2", ("fp64", "f32x2", "fp32")),
                                         ("film_128x64x2_descending.json", "film_128x64x2", ("fp64", "f32x2", "fp32")),
                                         ("film_512x256x4_descending.json", "film_512x256x4", ("fp64", "f32x2")))
         for p in precs]


def _stored(fname, workload):
    path = os.path.join(GOLDEN, fname)
    if not os.path.exists(path):
        pytest.skip(f"{fname} has not been stored")
    rec = json.load(open(path))
    spec = importlib.util.spec_from_file_location("make_oracle_loop", os.path.join(GOLDEN, "make_oracle_loop.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    w = inputs.WORKLOADS[workload]()
    assert rec["input_hash"] == mod.input_hash(w, w.initial_m(), w.fields()), "stored values are for other inputs"
    return w, rec


def _switches(b, p):
    """Index of the first descending value below zero field with p < 0, and
    of the first ascending value above zero field with p > 0 (None if absent)."""
    n = len(b)
    nd = 1
    while nd < n and b[nd] < b[nd - 1]:
        nd += 1
    down = next((i for i in range(nd) if b[i] < 0 and p[i] < 0), None)
    up = next((i for i in range(nd, n) if b[i] > 0 and p[i] > 0), None)
    return down, up, nd


@pytest.mark.parametrize("fname,workload,precision", CASES)
def test_loop_matches_oracle(mmlib, fname, workload, precision):
    w, rec = _stored(fname, workload)
    prec = {"fp64": mmlib.MM_FP64, "f32x2": mmlib.MM_F32X2, "fp32": mmlib.MM_FP32}[precision]
    H = np.array(rec["H"])
    n = len(H)
    assert n >= 2 and all(rec["converged"])
    grid = mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
    prob = mmlib.mm_setup_geometry(grid, mmlib.make_material(w.Ms, w.A, w.K), prec)
    m = dev(w.initial_m(), torch.float32 if precision == "fp32" else torch.float64)
    st, mavg, res = mmlib.mm_hysteresis_sweep(prob, m, H, opts=mmlib.make_opts(tol=w.tol, max_iter=rec["max_iter"]))
    prob.close()
    assert st == mmlib.MM_OK and all(r.converged for r in res)
    ref = np.array(rec["mavg"])
    hhat = inputs.field_direction(w.tilt_deg)
    b = np.array(rec["field_mT"])
    d_gpu, u_gpu, nd = _switches(b, mavg @ hhat)
    d_ref, u_ref, _ = _switches(b, ref @ hhat)
    print(fname, precision, "evaluations", sum(r.heff_evals for r in res), "oracle", sum(rec["heff_evals"]),
          "switch down", None if d_gpu is None else b[d_gpu], "oracle", None if d_ref is None else b[d_ref],
          "up", None if u_gpu is None else b[u_gpu], "oracle", None if u_ref is None else b[u_ref])
    if rec["complete"]:
        assert d_ref is not None and d_gpu is not None
        assert abs(b[d_gpu] - b[d_ref]) <= 1.0 + 1e-9          # one 1 mT field step
        if nd < n:                                                # the ascending branch is stored too
            assert u_ref is not None and u_gpu is not None
            assert abs(b[u_gpu] - b[u_ref]) <= 1.0 + 1e-9
    elif d_gpu is not None:
        # the stored branch ends before the oracle switched: the GPU must not switch earlier
        assert b[d_gpu] <= b[n - 1] + 1.0 + 1e-9
    zero = [i for i in range(nd) if abs(b[i]) < 1e-9]
    if zero:
        assert abs(mavg[zero[0], 0] - ref[zero[0], 0]) <= 1e-3
    # before the first switching event (a jump of <m> in either loop) both
    # follow the same minima
    first = n
    for mv in (mavg, ref):
        jump = np.nonzero(np.linalg.norm(np.diff(mv, axis=0), axis=1) > 0.02)[0]
        if len(jump):
            first = min(first, int(jump[0]) + 1)
    diff = np.max(np.abs(mavg[:first] - ref[:first]), axis=1)
    assert np.max(diff) < 1e-3, [(b[i], diff[i]) for i in np.nonzero(diff > 1e-3)[0]]
