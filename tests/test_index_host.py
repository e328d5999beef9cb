"""Index arithmetic of the field kernels, compiled for the host: the
multiply-shift divisor (FastDiv) against integer division, and the
shared-memory row layouts (a permutation into each row's slots, no overlap
between rows).  No GPU is used."""
import ctypes
import os
import random
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "idxh.so")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "index_host_harness.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.h_fastdiv_init.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int)]
    for n in ("h_spos_float", "h_spos_double"):
        getattr(L, n).argtypes = [ctypes.c_int]
    L.h_row_stride.argtypes = [ctypes.c_int, ctypes.c_int]
    return L


def fastdiv(L, d):
    mul, shift = ctypes.c_uint(), ctypes.c_int()
    L.h_fastdiv_init(d, ctypes.byref(mul), ctypes.byref(shift))
    m, s = mul.value, shift.value
    # the device quotient: (umulhi(n, mul) + n) >> shift in 32-bit unsigned arithmetic
    return lambda n: ((((n * m) >> 32) + n) & 0xFFFFFFFF) >> s


DIVISORS = [1, 2, 3, 5, 7, 31, 32, 33, 96, 100, 127, 255, 256, 257, 384, 511, 513, 1000, 1023, 1025, 2047, 2048,
            2049, 3000, 4095, 4096, 65535, 65537, 1 << 20, (1 << 20) + 1, 123456789]


@pytest.mark.parametrize("d", DIVISORS)
def test_fastdiv_equals_integer_division(lib, d):
    q = fastdiv(lib, d)
    rng = random.Random(d)
    ns = list(range(0, 4 * d + 5)) if d < 5000 else []
    for k in (1, 2, 3, 1000, 65536, (2**31 - 1) // d):
        ns += [k * d - 1, k * d, k * d + 1]
    ns += [2**31 - 1, 2**31 - 2, 2**30] + [rng.randrange(0, 2**31) for _ in range(20000)]
    for n in ns:
        if 0 <= n < 2**31:
            assert q(n) == n // d, (d, n)


LENGTHS = [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


@pytest.mark.parametrize("L", LENGTHS)
def test_float_rows_are_a_swizzle_within_groups_of_16(lib, L):
    pos = [lib.h_spos_float(i) for i in range(L)]
    stride = lib.h_row_stride(L, 8)
    assert stride == L + 1
    # a permutation of 0..L-1 that keeps every element in its aligned group of 16:
    # a row needs L slots and rows at stride L + 1 never overlap
    assert sorted(pos) == list(range(L))
    assert all(p >> 4 == i >> 4 for i, p in enumerate(pos))


@pytest.mark.parametrize("L", LENGTHS)
def test_double_rows_pad_one_slot_per_8(lib, L):
    pos = [lib.h_spos_double(i) for i in range(L)]
    stride = lib.h_row_stride(L, 16)
    assert pos == [i + (i >> 3) for i in range(L)]
    assert len(set(pos)) == L and max(pos) < stride


def test_float_swizzle_spreads_a_warp_over_all_banks(lib):
    # 16 consecutive float2 elements fill the 32 four-byte banks once each (one
    # wavefront); the swizzle keeps that for every aligned run of 16, and it
    # puts the 8 elements of a stride-16 column (bits 4-6 varying) in 8
    # distinct 8-byte bank pairs, where the plain layout puts them in one.
    for base in range(0, 4096, 16):
        slots = {lib.h_spos_float(base + j) % 16 for j in range(16)}
        assert len(slots) == 16
    for col in range(16):
        slots = [lib.h_spos_float(col + 16 * g) % 16 for g in range(8)]
        assert len(set(slots)) == 8
