"""CPU oracle for the energy-minimising hysteresis method (test infrastructure).

This package is the plain, slow reference that the CUDA library is checked
against.  It is test infrastructure only: the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the product library never does,
and it shares no code, tables or helpers with the CUDA path.

* ``newell_quad.c`` -- the Newell demagnetisation tensor in quadruple precision.
* ``micromag.py``   -- effective field, energy, the projected Barzilai-Borwein
  minimiser with the midpoint (Cayley) step, and the hysteresis sweep, in
  float64 numpy, following the paper's Section 2 step by step.
"""
