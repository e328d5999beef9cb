"""The stored oracle loops (tests/golden/*_loop.json, *_descending.json) are
the oracle's: re-running the committed script's steps with the oracle on the
first field values of the stored 128 x 64 x 2 loop reproduces the stored
<m> and evaluation counts (Section 4, the warm-started sweep; Section 2, the
minimiser).  This pins the expected values the GPU loop-parity tests use to
the oracle, not to the CUDA path."""
import importlib.util
import json
import os

import numpy as np

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _script():
    spec = importlib.util.spec_from_file_location("make_oracle_loop", os.path.join(GOLDEN, "make_oracle_loop.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stored_128x64x2_loop_starts_as_the_oracle_computes_it():
    rec = json.load(open(os.path.join(GOLDEN, "film_128x64x2_loop.json")))
    w = inputs.WORKLOADS["film_128x64x2"]()
    m0, H = w.initial_m(), w.fields()
    assert rec["input_hash"] == _script().input_hash(w, m0, H)
    prob = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K, u=w.u)
    demag = om.Demag(prob)
    m = m0
    for n in range(2):
        r = om.minimize(prob, m, H[n], demag, tol=w.tol, max_iter=rec["max_iter"])
        m = r.m
        mavg = m.reshape(3, -1).mean(axis=1)
        assert np.max(np.abs(mavg - np.array(rec["mavg"][n]))) <= 1e-12, n
        assert r.heff_evals == rec["heff_evals"][n], n
        assert bool(r.converged) and rec["converged"][n]
