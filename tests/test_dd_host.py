"""The library's double-double arithmetic (csrc/dd.cuh), compiled for the host,
against 60-digit multiprecision values (mpmath).  Checks the constants, the
elementary functions at dd accuracy and Newell's f and g at far-field
arguments, where the Newell tensor needs them."""
import ctypes
import os
import subprocess
import tempfile

import mpmath
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "ddh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                    os.path.join(HERE, "dd_host_harness.cpp"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    for name, n in (("h_exp", 2), ("h_log", 2), ("h_atan", 2), ("h_asinh", 2), ("h_sqrt", 2),
                    ("h_div", 4), ("h_f", 3), ("h_g", 3)):
        getattr(L, name).argtypes = [ctypes.c_double] * n + [dp]
    L.h_consts.argtypes = [dp]
    return L


def call(L, name, *args):
    out = (ctypes.c_double * 2)()
    getattr(L, name)(*[float(a) for a in args], out)
    return mpmath.mpf(out[0]) + mpmath.mpf(out[1])


def split(x):
    hi = float(x)
    return hi, float(x - mpmath.mpf(hi))


def test_constants(lib):
    mpmath.mp.dps = 60
    out = (ctypes.c_double * 4)()
    lib.h_consts(out)
    assert abs(mpmath.mpf(out[0]) + mpmath.mpf(out[1]) - mpmath.log(2)) < mpmath.mpf(2) ** -106
    assert abs(mpmath.mpf(out[2]) + mpmath.mpf(out[3]) - mpmath.pi) < mpmath.mpf(2) ** -104


@pytest.mark.parametrize("x", ["1e-9", "0.3", "0.6931471805599453", "1", "2.5", "-3.7", "17.25", "-40.5", "123.456"])
def test_exp_log(lib, x):
    mpmath.mp.dps = 60
    x = mpmath.mpf(x)
    hi, lo = split(x)
    xv = mpmath.mpf(hi) + mpmath.mpf(lo)
    e = call(lib, "h_exp", hi, lo)
    assert abs(e / mpmath.exp(xv) - 1) < mpmath.mpf(2) ** -100
    if x > 0:
        l = call(lib, "h_log", hi, lo)
        assert abs(l - mpmath.log(xv)) < mpmath.mpf(2) ** -100 * max(1, abs(mpmath.log(xv)))


@pytest.mark.parametrize("t", ["0", "1e-12", "0.01", "0.0625", "0.3", "1", "3.5", "1000", "1e8"])
def test_atan_asinh_sqrt(lib, t):
    mpmath.mp.dps = 60
    t = mpmath.mpf(t)
    hi, lo = split(t)
    tv = mpmath.mpf(hi) + mpmath.mpf(lo)
    a = call(lib, "h_atan", hi, lo)
    assert abs(a - mpmath.atan(tv)) <= mpmath.mpf(2) ** -103 * max(mpmath.mpf(1e-300), mpmath.atan(tv))
    s = call(lib, "h_asinh", hi, lo)
    assert abs(s - mpmath.asinh(tv)) <= mpmath.mpf(2) ** -102 * max(1, mpmath.asinh(tv))
    q = call(lib, "h_sqrt", hi, lo)
    assert abs(q - mpmath.sqrt(tv)) <= mpmath.mpf(2) ** -104 * max(mpmath.mpf(1e-300), mpmath.sqrt(tv))


def test_division(lib):
    mpmath.mp.dps = 60
    a, b = mpmath.mpf(1) / 3, mpmath.mpf(-7) / 11
    q = call(lib, "h_div", *split(a), *split(b))
    av = sum(mpmath.mpf(v) for v in split(a))
    bv = sum(mpmath.mpf(v) for v in split(b))
    assert abs(q / (av / bv) - 1) < mpmath.mpf(2) ** -104


def _f(x, y, z):
    x, y, z = abs(x), abs(y), abs(z)
    R = mpmath.sqrt(x * x + y * y + z * z)
    t = (2 * x * x - y * y - z * z) * R / 6
    if y > 0 and z * z != x * x:
        t += y / 2 * (z * z - x * x) * mpmath.asinh(y / mpmath.sqrt(x * x + z * z))
    if z > 0 and y * y != x * x:
        t += z / 2 * (y * y - x * x) * mpmath.asinh(z / mpmath.sqrt(x * x + y * y))
    if x > 0 and y > 0 and z > 0:
        t -= x * y * z * mpmath.atan(y * z / (x * R))
    return t


def _g(x, y, z):
    R = mpmath.sqrt(x * x + y * y + z * z)
    t = -x * y * R / 3
    if x > 0 and y > 0 and z > 0:
        t += x * y * z * mpmath.asinh(z / mpmath.sqrt(x * x + y * y))
        t -= z ** 3 / 6 * mpmath.atan(x * y / (z * R))
        t -= z * y * y / 2 * mpmath.atan(x * z / (y * R))
        t -= z * x * x / 2 * mpmath.atan(y * z / (x * R))
    if x > 0 and y > 0:
        t += y / 6 * (3 * z * z - y * y) * mpmath.asinh(x / mpmath.sqrt(y * y + z * z))
        t += x / 6 * (3 * z * z - x * x) * mpmath.asinh(y / mpmath.sqrt(x * x + z * z))
    return t


@pytest.mark.parametrize("p", [(0, 0, 0), (1, 0, 0), (0, 1, 2), (1, 1, 1), (3, 2, 1), (511.0, 255.0, 3.0),
                               (1000.0, 7.0, 2.0), (2.0, 0.78125, 0.5), (0.78125 * 400, 0.78125 * 200, 3.0)])
def test_newell_f_g_at_dd_accuracy(lib, p):
    mpmath.mp.dps = 60
    x, y, z = (mpmath.mpf(v) for v in p)
    scale = max(1, (x * x + y * y + z * z) ** 1.5)
    assert abs(call(lib, "h_f", *p) - _f(x, y, z)) <= mpmath.mpf(2) ** -100 * scale
    assert abs(call(lib, "h_g", *p) - _g(x, y, z)) <= mpmath.mpf(2) ** -100 * scale
