"""ctypes binding of libmmgb.so (include/mm.h), same names as the C entry points.

Argument marshalling only: every computation runs in the CUDA library.  Field
arguments are torch tensors (CUDA or CPU) or numpy arrays, contiguous, of shape
(3, nz, ny, nx) and the problem's dtype (float64 for MM_FP64, float32 for
MM_FP32).  PyTorch supplies device memory and streams; the library does the rest.

Importing this module loads the library and fails loudly if it has not been
built (``python -m paper_1405_2728_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_long, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmmgb.so")

MM_OK, MM_ERR_ARG, MM_ERR_OOM, MM_ERR_CUDA = 0, -1, -2, -3
MM_ERR_NOT_CONVERGED, MM_ERR_NONFINITE, MM_ERR_TIMEOUT, MM_ERR_UNSUPPORTED = -4, -5, -6, -7
MM_FP64, MM_FP32, MM_F32X2 = 0, 1, 2
MM_STEP_CAYLEY, MM_STEP_NORMALIZE = 0, 1
MM_TAU_ALTERNATE, MM_TAU_ADAPTIVE = 0, 1
MM_BATCH_AUTO, MM_BATCH_BRANCHES, MM_BATCH_GROUPED, MM_BATCH_STREAMS = 0, 1, 2, 3


class mm_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("dx", c_double), ("dy", c_double), ("dz", c_double)]


class mm_material(ctypes.Structure):
    _fields_ = [("Ms", c_double), ("A", c_double), ("K", c_double), ("u", c_double * 3),
                ("K_cell", c_void_p), ("u_cell", c_void_p)]


class mm_min_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("tau0", c_double), ("max_iter", c_long), ("step_kind", c_int),
                ("timeout_s", c_double), ("tau_rule", c_int), ("tau_kappa", c_double)]


class mm_min_result(ctypes.Structure):
    _fields_ = [("iters", c_long), ("heff_evals", c_long), ("max_torque", c_double), ("energy", c_double),
                ("converged", c_int), ("status", c_int), ("kernel_launches", c_long)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mm_info(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("px", c_int), ("py", c_int), ("pz", c_int),
                ("precision", c_int), ("cells", c_long), ("workspace_bytes", c_long),
                ("spectrum_bytes", c_long), ("tensor_bytes", c_long), ("x_tile_rows", c_int),
                ("yz_batch_rows", c_int), ("bulk_layout", c_int),
                ("x_fwd_tile_rows", c_int)]


class mm_min_state(ctypes.Structure):
    _fields_ = [("k", c_long), ("status", c_int), ("tau", c_double), ("ss", c_double), ("sy", c_double),
                ("yy", c_double), ("max_torque", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = f"{where}: {mm_status_string(status)} ({status})"
        if status == MM_ERR_CUDA:
            msg += f" [{mm_last_cuda_error()}]"
        super().__init__(msg)


_lib = None


def lib():
    """The loaded libmmgb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmmgb.so not found at {LIB_PATH}: build it first "
                              "(python -m paper_1405_2728_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        dp = POINTER(c_double)
        L.mm_newell.argtypes = [POINTER(mm_grid), c_void_p, c_void_p]
        L.mm_newell_static.argtypes = [POINTER(mm_grid), c_void_p, c_void_p]
        L.mm_setup_geometry.argtypes = [POINTER(mm_grid), POINTER(mm_material), c_int, c_void_p, POINTER(c_void_p)]
        L.mm_destroy.argtypes = [c_void_p]
        L.mm_heff.argtypes = [c_void_p, c_void_p, dp, c_void_p, c_void_p]
        L.mm_energy.argtypes = [c_void_p, c_void_p, dp, dp, c_void_p]
        L.mm_minimize.argtypes = [c_void_p, c_void_p, dp, POINTER(mm_min_opts), POINTER(mm_min_result), c_void_p]
        L.mm_hysteresis_sweep.argtypes = [c_void_p, c_void_p, dp, c_int, c_int, POINTER(mm_min_opts), dp,
                                          POINTER(mm_min_result), c_void_p]
        L.mm_problem_info.argtypes = [c_void_p, POINTER(mm_info)]
        L.mm_kernel_times.argtypes = [c_void_p, c_void_p, dp, c_int, dp, POINTER(c_char_p), POINTER(c_int), c_void_p]
        L.mm_energy_gradient.argtypes = [c_void_p, c_void_p, dp, c_double, c_void_p, c_void_p]
        L.mm_hessian_vec.argtypes = [c_void_p, c_void_p, dp, c_void_p, c_void_p, c_void_p]
        L.mm_adjoint_dK.argtypes = [c_void_p, c_void_p, dp, c_void_p, c_void_p, c_double, c_long,
                                    POINTER(c_long), POINTER(c_double), c_void_p]
        L.mm_set_anisotropy.argtypes = [c_void_p, c_void_p, c_void_p]
        L.mm_hysteresis_sweep_mixed.argtypes = [c_void_p, c_void_p, c_void_p, dp, c_int, c_int,
                                                POINTER(mm_min_opts), POINTER(mm_min_opts), dp,
                                                POINTER(mm_min_result), POINTER(mm_min_result), c_void_p]
        L.mm_probe_fma.argtypes = [dp]
        L.mm_min_inspect.argtypes = [c_void_p, POINTER(mm_min_state), c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]
        L.mm_batch_create.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p)]
        L.mm_batch_create_kind.argtypes = [POINTER(c_void_p), c_int, c_int, POINTER(c_void_p)]
        L.mm_batch_kind.argtypes = [c_void_p]
        L.mm_batch_destroy.argtypes = [c_void_p]
        L.mm_batch_sweep.argtypes = [c_void_p, POINTER(c_void_p), dp, c_int, c_int, POINTER(mm_min_opts), dp,
                                     POINTER(mm_min_result), c_void_p]
        L.mm_status_string.argtypes = [c_int]
        L.mm_status_string.restype = c_char_p
        L.mm_last_cuda_error.restype = c_char_p
        for name in ("mm_newell", "mm_newell_static", "mm_setup_geometry", "mm_destroy", "mm_heff", "mm_energy", "mm_minimize",
                     "mm_hysteresis_sweep", "mm_problem_info", "mm_kernel_times", "mm_energy_gradient",
                     "mm_hessian_vec", "mm_adjoint_dK", "mm_set_anisotropy", "mm_hysteresis_sweep_mixed", "mm_batch_create",
                     "mm_batch_create_kind", "mm_batch_kind", "mm_batch_destroy", "mm_batch_sweep", "mm_probe_fma", "mm_min_inspect"):
            getattr(L, name).restype = c_int
        _lib = L
    return _lib


def mm_status_string(status: int) -> str:
    return lib().mm_status_string(int(status)).decode()


def mm_last_cuda_error() -> str:
    return lib().mm_last_cuda_error().decode()


def _check(status, where):
    if status != MM_OK:
        raise MMError(status, where)


# --- argument marshalling ---------------------------------------------------

def _ptr(a, dtype=None, shape=None, what="array"):
    """Raw data pointer of a contiguous torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):  # torch.Tensor
        if not a.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if dtype is not None and str(a.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"{what} has dtype {a.dtype}, expected {np.dtype(dtype).name}")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"{what} has shape {tuple(a.shape)}, expected {tuple(shape)}")
        return c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what} must be C-contiguous")
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise TypeError(f"{what} has dtype {a.dtype}, expected {np.dtype(dtype).name}")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"{what} has shape {tuple(a.shape)}, expected {tuple(shape)}")
        return c_void_p(a.ctypes.data)
    raise TypeError(f"{what}: expected a torch tensor or numpy array, got {type(a).__name__}")


def _stream(stream, *arrays):
    """cudaStream_t handle: explicit int/torch stream, else torch's current stream
    when a CUDA tensor is involved, else the legacy default stream (0)."""
    if stream is not None:
        return c_void_p(int(getattr(stream, "cuda_stream", stream)))
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return c_void_p(0)


def _mavg(mavg, n):
    """Per-field <m> output that the library writes on the host: a writable,
    C-contiguous float64 numpy array (n, 3); a new one (NaN) when None."""
    if mavg is None:
        return np.full((n, 3), np.nan)
    if (not isinstance(mavg, np.ndarray) or mavg.dtype != np.float64 or mavg.shape != (n, 3)
            or not mavg.flags["C_CONTIGUOUS"] or not mavg.flags["WRITEABLE"]):
        raise ValueError(f"mavg must be a writable C-contiguous float64 numpy array of shape ({n}, 3)")
    return mavg


def _vec3(h):
    v = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(3))
    return v, v.ctypes.data_as(POINTER(c_double))


# --- problem ------------------------------------------------------------------

class Problem:
    """Owner of an mm_problem*; destroyed with mm_destroy."""

    def __init__(self, handle, grid, precision):
        self.handle = handle
        self.grid = grid
        self.precision = precision
        self.dtype = np.float32 if precision == MM_FP32 else np.float64
        self.shape = (3, grid.nz, grid.ny, grid.nx)

    def close(self):
        if self.handle:
            lib().mm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_grid(nx, ny, nz, dx, dy, dz) -> mm_grid:
    return mm_grid(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz))


def make_material(Ms, A, K=0.0, u=(1.0, 0.0, 0.0), K_cell=None, u_cell=None) -> mm_material:
    mat = mm_material(float(Ms), float(A), float(K), (c_double * 3)(*[float(x) for x in u]), None, None)
    mat._keep = []
    if K_cell is not None:
        mat.K_cell = _ptr(K_cell, np.float64, what="K_cell").value
        mat._keep.append(K_cell)
    if u_cell is not None:
        mat.u_cell = _ptr(u_cell, np.float64, what="u_cell").value
        mat._keep.append(u_cell)
    return mat


def make_opts(tol=1e-5, tau0=0.0, max_iter=100000, step_kind=MM_STEP_CAYLEY, timeout_s=0.0,
              tau_rule=MM_TAU_ALTERNATE, tau_kappa=0.0) -> mm_min_opts:
    return mm_min_opts(float(tol), float(tau0), int(max_iter), int(step_kind), float(timeout_s), int(tau_rule),
                       float(tau_kappa))


def mm_newell(grid: mm_grid, N_out, stream=None):
    """Newell tensor octant into N_out (6, nz, ny, nx) float64 (host or device)."""
    _check(lib().mm_newell(ctypes.byref(grid), _ptr(N_out, np.float64, (6, grid.nz, grid.ny, grid.nx), "N_out"),
                           _stream(stream, N_out)), "mm_newell")
    return N_out


def mm_newell_static(grid: mm_grid, N_out, stream=None):
    """As mm_newell, without device allocation: N_out must be a CUDA tensor
    (6, nz, ny, nx) float64; asynchronous on the stream; grids up to
    (nx+1)(ny+1)(nz+1) <= 65536 lattice points."""
    _check(lib().mm_newell_static(ctypes.byref(grid),
                                  _ptr(N_out, np.float64, (6, grid.nz, grid.ny, grid.nx), "N_out"),
                                  _stream(stream, N_out)), "mm_newell_static")
    return N_out


def mm_setup_geometry(grid: mm_grid, mat: mm_material, precision=MM_FP64, stream=None) -> Problem:
    h = c_void_p()
    _check(lib().mm_setup_geometry(ctypes.byref(grid), ctypes.byref(mat), int(precision), _stream(stream),
                                   ctypes.byref(h)), "mm_setup_geometry")
    return Problem(h, grid, precision)


def mm_destroy(prob: Problem):
    prob.close()


def mm_heff(prob: Problem, m, Hext, H_out, stream=None):
    h = _vec3(Hext)
    _check(lib().mm_heff(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1],
                         _ptr(H_out, prob.dtype, prob.shape, "H_out"), _stream(stream, m, H_out)), "mm_heff")
    return H_out


def mm_energy(prob: Problem, m, Hext, stream=None) -> np.ndarray:
    """Energy terms (demag, exchange, anisotropy, zeeman, total) in J."""
    h = _vec3(Hext)
    E = np.zeros(5)
    _check(lib().mm_energy(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1],
                           E.ctypes.data_as(POINTER(c_double)), _stream(stream, m)), "mm_energy")
    return E


_SOFT = (MM_OK, MM_ERR_NOT_CONVERGED, MM_ERR_NONFINITE, MM_ERR_TIMEOUT)


def mm_minimize(prob: Problem, m, Hext, opts: mm_min_opts | None = None, stream=None):
    """Minimise in place; returns (status, mm_min_result).  Raises on argument/CUDA errors."""
    opts = opts or make_opts()
    h = _vec3(Hext)
    res = mm_min_result()
    st = lib().mm_minimize(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1], ctypes.byref(opts),
                           ctypes.byref(res), _stream(stream, m))
    if st not in _SOFT:
        raise MMError(st, "mm_minimize")
    return st, res


def mm_hysteresis_sweep(prob: Problem, m, H_list, start=0, opts: mm_min_opts | None = None, stream=None,
                        mavg=None):
    """Run the sweep over H_list (n, 3) A/m; returns (status, mavg (n,3), [mm_min_result])."""
    opts = opts or make_opts()
    H = np.ascontiguousarray(np.asarray(H_list, dtype=np.float64).reshape(-1, 3))
    n = H.shape[0]
    mavg = _mavg(mavg, n)
    res = (mm_min_result * n)()
    st = lib().mm_hysteresis_sweep(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"),
                                   H.ctypes.data_as(POINTER(c_double)), n, int(start), ctypes.byref(opts),
                                   mavg.ctypes.data_as(POINTER(c_double)), res, _stream(stream, m))
    if st not in _SOFT:
        raise MMError(st, "mm_hysteresis_sweep")
    return st, mavg, list(res)


def mm_hysteresis_sweep_mixed(lo: Problem, hi: Problem, m, H_list, start=0, opts_lo: mm_min_opts | None = None,
                              opts_hi: mm_min_opts | None = None, stream=None, mavg=None):
    """Mixed-precision sweep: per field value an FP32 minimisation (opts_lo,
    loose tolerance) then one of hi's precision, FP64 or double-word (opts_hi).
    m is float64 [3][nz][ny][nx].  The default hand-over tolerance is the
    fastest measured on the 512x256x4 film: 3e-5 before FP64, 1e-4 before
    double-word.  Returns (status, mavg (n,3), [FP32 results], [hi results])."""
    if opts_lo is None:
        opts_lo = make_opts(tol=1e-4 if hi.precision == MM_F32X2 else 3e-5, max_iter=20000)
    opts_hi = opts_hi or make_opts()
    H = np.ascontiguousarray(np.asarray(H_list, dtype=np.float64).reshape(-1, 3))
    n = H.shape[0]
    mavg = _mavg(mavg, n)
    rl, rh = (mm_min_result * n)(), (mm_min_result * n)()
    st = lib().mm_hysteresis_sweep_mixed(lo.handle, hi.handle, _ptr(m, np.float64, hi.shape, "m"),
                                         H.ctypes.data_as(POINTER(c_double)), n, int(start), ctypes.byref(opts_lo),
                                         ctypes.byref(opts_hi), mavg.ctypes.data_as(POINTER(c_double)), rl, rh,
                                         _stream(stream, m))
    if st not in _SOFT:
        raise MMError(st, "mm_hysteresis_sweep_mixed")
    return st, mavg, list(rl), list(rh)


def mm_problem_info(prob: Problem) -> dict:
    info = mm_info()
    _check(lib().mm_problem_info(prob.handle, ctypes.byref(info)), "mm_problem_info")
    return {f: getattr(info, f) for f, _ in info._fields_}


def mm_kernel_times(prob: Problem, m, Hext, reps=20, stream=None) -> dict:
    """Average device time (ms) of each kernel stage of one minimiser iteration."""
    h = _vec3(Hext)
    ms = (c_double * 16)()
    names = (c_char_p * 16)()
    cnt = c_int(16)
    _check(lib().mm_kernel_times(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1], int(reps), ms, names,
                                 ctypes.byref(cnt), _stream(stream, m)), "mm_kernel_times")
    return {names[i].decode(): ms[i] for i in range(cnt.value)}


def mm_min_inspect(prob: Problem, m_k=None, m_prev=None, g_k=None, g_prev=None, stream=None) -> dict:
    """State of the last minimisation (iterate index, step size, BB sums, torque,
    status); optional arrays receive m_k, m_{k-1}, g_k, g_{k-1}."""
    out = mm_min_state()
    bufs = [None if a is None else _ptr(a, prob.dtype, prob.shape, "buffer") for a in (m_k, m_prev, g_k, g_prev)]
    _check(lib().mm_min_inspect(prob.handle, ctypes.byref(out), *bufs,
                                _stream(stream, *[a for a in (m_k, m_prev, g_k, g_prev) if a is not None])),
           "mm_min_inspect")
    return out.as_dict()


def mm_probe_fma() -> dict:
    """Measured FMA throughput of the current device (TFLOP/s): {"fp64": .., "fp32": ..}."""
    out = (c_double * 2)()
    _check(lib().mm_probe_fma(out), "mm_probe_fma")
    return {"fp64": out[0], "fp32": out[1]}


def mm_energy_gradient(prob: Problem, m, Hext, G_out, scale=1.0, stream=None):
    """G_out = scale * dU/dm = -scale * mu0 Ms V H_eff(m)."""
    h = _vec3(Hext)
    _check(lib().mm_energy_gradient(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1], float(scale),
                                    _ptr(G_out, prob.dtype, prob.shape, "G_out"), _stream(stream, m, G_out)),
           "mm_energy_gradient")
    return G_out


def mm_hessian_vec(prob: Problem, m, Hext, v, Av, stream=None):
    """Av = (m.H) v - P_m(L v) for a tangent field v."""
    h = _vec3(Hext)
    _check(lib().mm_hessian_vec(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1],
                                _ptr(v, prob.dtype, prob.shape, "v"), _ptr(Av, prob.dtype, prob.shape, "Av"),
                                _stream(stream, m, v, Av)), "mm_hessian_vec")
    return Av


def mm_adjoint_dK(prob: Problem, m, Hext, dJdm, dJdK, tol=1e-10, max_iter=10000, stream=None):
    """dJ/dK per cell at a converged minimum; returns (status, iterations, relative residual)."""
    h = _vec3(Hext)
    it = c_long(0)
    res = c_double(0.0)
    st = lib().mm_adjoint_dK(prob.handle, _ptr(m, prob.dtype, prob.shape, "m"), h[1],
                             _ptr(dJdm, prob.dtype, prob.shape, "dJdm"),
                             _ptr(dJdK, np.float64, prob.shape[1:], "dJdK"), float(tol), int(max_iter),
                             ctypes.byref(it), ctypes.byref(res), _stream(stream, m, dJdm, dJdK))
    if st not in _SOFT:
        raise MMError(st, "mm_adjoint_dK")
    return st, it.value, res.value


def mm_set_anisotropy(prob: Problem, K_cell, stream=None):
    """Replace the per-cell K (float64 (nz, ny, nx), host or device)."""
    _check(lib().mm_set_anisotropy(prob.handle, _ptr(K_cell, np.float64, prob.shape[1:], "K_cell"),
                                   _stream(stream, K_cell)), "mm_set_anisotropy")


class Batch:
    """Owner of an mm_batch*; keeps its problems alive."""

    def __init__(self, handle, probs):
        self.handle = handle
        self.probs = list(probs)

    def close(self):
        if self.handle:
            lib().mm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mm_batch_create(probs, kind=None) -> Batch:
    """A batch over probs; kind one of MM_BATCH_AUTO (default: the branch
    graph), MM_BATCH_BRANCHES, MM_BATCH_GROUPED, MM_BATCH_STREAMS."""
    arr = (c_void_p * len(probs))(*[p.handle for p in probs])
    h = c_void_p()
    _check(lib().mm_batch_create_kind(arr, len(probs), MM_BATCH_AUTO if kind is None else int(kind), ctypes.byref(h)),
           "mm_batch_create_kind")
    return Batch(h, probs)


def mm_batch_kind(batch: Batch) -> int:
    return lib().mm_batch_kind(batch.handle)


def mm_batch_destroy(batch: Batch):
    batch.close()


def mm_batch_sweep(batch: Batch, m_list, H_list, start=0, opts: mm_min_opts | None = None, stream=None):
    """Sweep every problem of the batch over H_list (n, 3); returns
    (status, mavg (nprob, n, 3), per_step results [nprob][n])."""
    opts = opts or make_opts()
    H = np.ascontiguousarray(np.asarray(H_list, dtype=np.float64).reshape(-1, 3))
    n = H.shape[0]
    P = len(batch.probs)
    if len(m_list) != P:
        raise ValueError(f"m_list has {len(m_list)} fields for {P} problems")
    ptrs = (c_void_p * P)(*[_ptr(m, p.dtype, p.shape, "m") for m, p in zip(m_list, batch.probs)])
    mavg = np.full((P, n, 3), np.nan)
    res = (mm_min_result * (P * n))()
    st = lib().mm_batch_sweep(batch.handle, ptrs, H.ctypes.data_as(POINTER(c_double)), n, int(start),
                              ctypes.byref(opts), mavg.ctypes.data_as(POINTER(c_double)), res,
                              _stream(stream, *m_list))
    if st not in _SOFT:
        raise MMError(st, "mm_batch_sweep")
    return st, mavg, [list(res[i * n:(i + 1) * n]) for i in range(P)]
