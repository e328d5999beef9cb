"""Compile the quad-precision Newell oracle (``newell_quad.c``) with gcc.

Test infrastructure: builds ``oracle/_newell_quad.so`` next to this file.
x86-64 links libquadmath (``__float128``); aarch64 uses binary128
``long double`` from libm.  OpenMP parallelises the tensor tabulation.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "newell_quad.c")
LIB = os.path.join(HERE, "_newell_quad.so")


def build(force: bool = False) -> str:
    """Build the shared library if missing or older than its source; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", SRC, "-o", LIB + ".tmp", "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
