"""mm_newell_static: the Newell tensor for callers that cannot allocate.

Callers whose device memory is already reserved by another allocator, or that
run on streams where cudaMalloc/cudaFree (device-wide synchronisation) are not
allowed, use this entry point; its work table is a static device array that
every call shares.  It must give what mm_newell gives.  Two static calls in a
row on the same stream, the second on a smaller grid, check that the second
call is ordered after the first and that the shared table carries nothing
over from it.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
CELL = (3.90625e-9, 3.90625e-9, 5e-9)


def _static(mmlib, shape, stream):
    nx, ny, nz = shape
    grid = mmlib.make_grid(nx, ny, nz, *CELL)
    got = torch.full((6, nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    rc = mmlib.lib().mm_newell_static(ctypes.byref(grid), ctypes.c_void_p(got.data_ptr()),
                                      ctypes.c_void_p(stream))
    assert rc == mmlib.MM_OK, mmlib.mm_status_string(rc)
    return got


def _reference(mmlib, shape):
    nx, ny, nz = shape
    ref = torch.zeros((6, nz, ny, nx), dtype=torch.float64, device="cuda")
    mmlib.mm_newell(mmlib.make_grid(nx, ny, nz, *CELL), ref)
    return ref.cpu().numpy()


def _check(got, ref):
    g = got.cpu().numpy()
    assert np.all(np.isfinite(g))
    # same tolerance as the tensor parity tests (and in practice identical bits)
    assert np.max(np.abs(g - ref)) <= 2e-15 * np.abs(ref).max()


def test_static_scratch_newell_matches_mm_newell(mmlib):
    stream = torch.cuda.current_stream().cuda_stream
    for shape in [(40, 20, 3), (7, 5, 2), (255, 127, 1)]:
        ref = _reference(mmlib, shape)
        got = _static(mmlib, shape, stream)
        torch.cuda.synchronize()
        _check(got, ref)


def test_two_static_calls_in_a_row_on_one_stream(mmlib):
    """The large grid fills most of the shared table; the small grid's call,
    issued right after it with no host synchronisation in between, must still
    equal mm_newell (work on one stream is ordered)."""
    refs = {s: _reference(mmlib, s) for s in [(255, 127, 1), (7, 5, 2)]}
    stream = torch.cuda.current_stream().cuda_stream
    big = _static(mmlib, (255, 127, 1), stream)
    small = _static(mmlib, (7, 5, 2), stream)
    torch.cuda.synchronize()
    _check(big, refs[(255, 127, 1)])
    _check(small, refs[(7, 5, 2)])


def test_static_scratch_rejects_oversize_and_host_buffers(mmlib):
    lib = mmlib.lib()
    big = mmlib.make_grid(256, 128, 1, *CELL)   # 257*129*2 > 65536 lattice points
    out = torch.zeros((6, 1, 128, 256), dtype=torch.float64, device="cuda")
    assert lib.mm_newell_static(ctypes.byref(big), ctypes.c_void_p(out.data_ptr()), None) == mmlib.MM_ERR_UNSUPPORTED
    small = mmlib.make_grid(4, 4, 1, *CELL)
    host = np.zeros((6, 1, 4, 4))
    assert lib.mm_newell_static(ctypes.byref(small), ctypes.c_void_p(host.ctypes.data), None) == mmlib.MM_ERR_ARG
