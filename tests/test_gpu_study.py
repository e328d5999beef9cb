"""SP1 convergence study (Section 4) through the library, on the 10 nm grid:
the loops converge at every field value, the metrics are well defined, and
halving the field step moves the coercive field by less than the coarse
step (the paper's statement that 0.5 mT steps do not change the loop).  The
field runs along the short edge: there the loop has no branch point whose
choice rounding could decide (along the long edge the first reversal of a
finer grid does depend on the field step)."""
import numpy as np
import pytest

from paper_1405_2728_gb300 import inputs, study

pytestmark = pytest.mark.gpu


def test_sp1_10nm_step_halving_short_edge(mmlib):
    out = {}
    for step in (1.0, 0.5):
        met, rem, evals, sec = study.run_loop(10.0, step, "short", mmlib.MM_FP64)
        assert met["converged"] and met["grid"] == [200, 100, 2]
        assert met["H_sw"] is not None and met["M_r"] is not None
        hc = met["H_c"] * inputs.MU0 * 1e3
        assert -50.0 < hc < 0.0
        assert abs(met["M_r"][0]) <= 1.0
        assert np.allclose(np.linalg.norm(rem, axis=0), 1.0, atol=1e-12)
        out[step] = hc
    assert abs(out[1.0] - out[0.5]) <= 1.0, out
