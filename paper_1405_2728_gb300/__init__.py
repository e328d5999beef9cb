"""GB300-native energy-minimising hysteresis solver for finite-difference micromagnetics.

The compute path lives in the CUDA library ``libmmgb.so`` (built from
``csrc/`` for sm_103a); ``mm`` is its thin ctypes binding and ``inputs``
generates seeded synthetic workloads.  Importing this package loads nothing.
"""
__all__ = ["mm", "inputs"]
__version__ = "0.1.0"
