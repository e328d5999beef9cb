"""mm_newell_static: the Newell tensor for callers that cannot allocate.

Callers whose device memory is already reserved by another allocator, or that
run on streams where cudaMalloc/cudaFree (device-wide synchronisation) are not
allowed, use this entry point; its work table is a static device array.  It
must give what mm_newell gives.  Two calls in a row on different grids check
that the shared table carries nothing over from the previous call.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
CELL = (3.90625e-9, 3.90625e-9, 5e-9)


def test_static_scratch_newell_matches_mm_newell(mmlib):
    lib = mmlib.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for (nx, ny, nz) in [(40, 20, 3), (7, 5, 2), (255, 127, 1)]:
        grid = mmlib.make_grid(nx, ny, nz, *CELL)
        ref = torch.zeros((6, nz, ny, nx), dtype=torch.float64, device="cuda")
        mmlib.mm_newell(grid, ref)
        got = torch.full((6, nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.mm_newell_static(ctypes.byref(grid), ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(stream))
        assert rc == mmlib.MM_OK, mmlib.mm_status_string(rc)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        # same tolerance as the tensor parity tests (and in practice identical bits)
        assert np.max(np.abs(g - r)) <= 2e-15 * np.abs(r).max()


def test_static_scratch_rejects_oversize_and_host_buffers(mmlib):
    lib = mmlib.lib()
    big = mmlib.make_grid(256, 128, 1, *CELL)   # 257*129*2 > 65536 lattice points
    out = torch.zeros((6, 1, 128, 256), dtype=torch.float64, device="cuda")
    assert lib.mm_newell_static(ctypes.byref(big), ctypes.c_void_p(out.data_ptr()), None) == mmlib.MM_ERR_UNSUPPORTED
    small = mmlib.make_grid(4, 4, 1, *CELL)
    host = np.zeros((6, 1, 4, 4))
    assert lib.mm_newell_static(ctypes.byref(small), ctypes.c_void_p(host.ctypes.data), None) == mmlib.MM_ERR_ARG
