"""ctypes binding of libmotjvie (argument marshalling only).

Every function keeps the C name and argument order of include/motjvie.h; device
arrays are passed as raw pointers (``int``) or as torch CUDA tensors, host arrays
as numpy arrays.  Errors raise MotError carrying the library's message.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmotjvie.so")

MOT_OK = 0
MOT_EINVAL = -1
MOT_ENOMEM = -2
MOT_ENOTCONV = -3
MOT_EUNSUPPORTED = -4
MOT_ECUDA = -5
MOT_ETIMEOUT = -6
MOT_EBUSY = -7
MOT_ECANCELLED = -8
MOT_FP64 = 0
MOT_MIXED = 1
MOT_FP64DF = 2
MOT_F64 = 0
MOT_F32 = 1
MOT_F64DF = 2
MOT_STATIC_SCRATCH_BYTES = 64 << 20

__all__ = [
    "LIB_PATH", "MotError", "lib", "mot_planewave", "mot_options", "mot_problem_info", "mot_step_stats",
    "mot_last_error", "mot_ctx_create", "mot_ctx_destroy", "mot_problem_create", "mot_problem_info_get",
    "mot_problem_destroy", "mot_apply_Z0", "mot_kernel_table", "mot_set_kernel_table", "mot_table_host",
    "mot_run_create", "mot_run_step", "mot_run_current_device", "mot_run_step_index", "mot_run_destroy",
    "MOT_OK", "MOT_EINVAL", "MOT_ENOMEM", "MOT_ENOTCONV", "MOT_EUNSUPPORTED", "MOT_ECUDA", "MOT_ETIMEOUT",
    "MOT_FP64", "MOT_MIXED", "MOT_FP64DF", "MOT_F64", "MOT_F32", "MOT_F64DF", "EXPORTED", "mot_kernel_launches", "default_options",
    "mot_apply_Z0_static", "MOT_STATIC_SCRATCH_BYTES", "mot_run_kernel_times", "KERNEL_CLASSES",
    "mot_run_save", "mot_run_load", "MOT_EBUSY", "MOT_ECANCELLED", "mot_request", "mot_result",
    "mot_server_create", "mot_server_submit", "mot_server_wait", "mot_server_destroy", "mot_fma_peak",
    "mot_schedule", "mot_problem_schedule", "mot_apply_Z0_direct",
]

# every symbol include/motjvie.h declares
EXPORTED = [
    "mot_last_error", "mot_ctx_create", "mot_ctx_destroy", "mot_problem_create", "mot_problem_info_get",
    "mot_problem_destroy", "mot_apply_Z0", "mot_kernel_table", "mot_set_kernel_table", "mot_table_host",
    "mot_run_create", "mot_run_step", "mot_run_current_device", "mot_run_step_index", "mot_run_destroy",
    "mot_kernel_launches", "mot_apply_Z0_static", "mot_run_kernel_times", "mot_run_save", "mot_run_load",
    "mot_server_create", "mot_server_submit", "mot_server_wait", "mot_server_destroy", "mot_fma_peak",
    "mot_problem_schedule", "mot_apply_Z0_direct",
]

# mot_kernel_class values, in order
KERNEL_CLASSES = ["z_green", "z_history", "fwd_half", "fwd_y1", "fwd_plain", "fwd_ring", "inv_half", "inv_v",
                  "inv_z0", "inv_residual", "inv_history", "row_fwd", "row_inv", "vec", "hist_side"]


class MotError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmotjvie status {status}: {msg}")
        self.status = status


class mot_planewave(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("sigma", ctypes.c_double), ("t0", ctypes.c_double),
                ("f0", ctypes.c_double), ("khat", ctypes.c_double * 3), ("pol", ctypes.c_double * 3)]


class mot_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("delta", ctypes.c_double), ("timing", ctypes.c_int),
                ("guess", ctypes.c_int), ("graph", ctypes.c_int), ("autotune", ctypes.c_int)]


class mot_schedule(ctypes.Structure):
    _fields_ = [("z_cols", ctypes.c_int32), ("x_rows", ctypes.c_int32), ("xy_fwd", ctypes.c_int32),
                ("xy_inv", ctypes.c_int32), ("pdl", ctypes.c_int32), ("gen_pairs", ctypes.c_int32),
                ("gen_tile", ctypes.c_int32), ("z_tma", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("rejected", ctypes.c_int32),
                ("cached", ctypes.c_int32), ("ms_default", ctypes.c_float), ("ms_tuned", ctypes.c_float),
                ("max_rel_diff", ctypes.c_double)]


class mot_problem_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("M0", ctypes.c_int32 * 3), ("Mh", ctypes.c_int32 * 3),
                ("r0", ctypes.c_int32), ("ell", ctypes.c_int32), ("rho", ctypes.c_double), ("dt", ctypes.c_double)]


class mot_step_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("relres", ctypes.c_double),
                ("ms_history", ctypes.c_float), ("ms_solve", ctypes.c_float), ("ms_push", ctypes.c_float),
                ("mvps", ctypes.c_int32), ("ms_zhist", ctypes.c_float), ("ms_zgreen", ctypes.c_float)]


class mot_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("h", ctypes.c_double), ("eps_r", ctypes.c_void_p),
                ("alpha", ctypes.c_double), ("precision", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("exc", ctypes.c_void_p), ("nsteps", ctypes.c_int32), ("opt", ctypes.c_void_p),
                ("J_final", ctypes.c_void_p)]


class mot_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("step_p50_ms", ctypes.c_float), ("step_p99_ms", ctypes.c_float),
                ("device_bytes", ctypes.c_uint64)]


_lib = None


def lib():
    """Load libmotjvie.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MotError(MOT_ECUDA, f"{LIB_PATH} not built (run paper_2607_28309_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        PP = ctypes.POINTER(ctypes.c_void_p)
        L.mot_last_error.restype = ctypes.c_char_p
        L.mot_ctx_create.argtypes = [I, P, PP]
        L.mot_ctx_destroy.argtypes = [P]
        L.mot_ctx_destroy.restype = None
        L.mot_problem_create.argtypes = [P, P, D, P, D, P, PP]
        L.mot_problem_info_get.argtypes = [P, P]
        L.mot_problem_destroy.argtypes = [P]
        L.mot_problem_destroy.restype = None
        L.mot_apply_Z0.argtypes = [P, P, P, I, I]
        L.mot_apply_Z0_static.argtypes = [P, P, P, I, I]
        L.mot_apply_Z0_direct.argtypes = [P, P, P, I, I]
        L.mot_kernel_table.argtypes = [P, I, P, P]
        L.mot_set_kernel_table.argtypes = [P, I, P, P]
        L.mot_table_host.argtypes = [D, I, P, P]
        L.mot_run_create.argtypes = [P, I, P, I, PP]
        L.mot_run_step.argtypes = [P, I, P, P]
        L.mot_run_current_device.argtypes = [P, PP]
        L.mot_run_step_index.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.mot_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.mot_run_kernel_times.argtypes = [P, I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]
        L.mot_run_save.argtypes = [P, ctypes.c_char_p]
        L.mot_server_create.argtypes = [P, ctypes.c_size_t, I, PP]
        L.mot_server_submit.argtypes = [P, ctypes.POINTER(mot_request), ctypes.POINTER(ctypes.c_uint64)]
        L.mot_server_wait.argtypes = [P, ctypes.c_uint64, D, ctypes.POINTER(mot_result)]
        L.mot_server_destroy.argtypes = [P]
        L.mot_server_destroy.restype = None
        L.mot_run_load.argtypes = [P, ctypes.c_char_p, PP]
        L.mot_fma_peak.argtypes = [I, I, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.mot_problem_schedule.argtypes = [P, I, I, ctypes.POINTER(mot_schedule)]
        L.mot_run_destroy.argtypes = [P]
        L.mot_run_destroy.restype = None
        for name in EXPORTED:
            if name not in ("mot_ctx_destroy", "mot_problem_destroy", "mot_run_destroy", "mot_last_error",
                            "mot_server_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != MOT_OK:
        raise MotError(status, mot_last_error())


def _ptr(a):
    """device pointer of a torch tensor / int, or host pointer of a numpy array"""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def mot_last_error() -> str:
    return lib().mot_last_error().decode()


def mot_ctx_create(device: int = 0, cuda_stream: int | None = None):
    out = ctypes.c_void_p()
    # cuda_stream None or 0: the legacy default stream (PyTorch's default stream)
    _check(lib().mot_ctx_create(int(device), ctypes.c_void_p(cuda_stream) if cuda_stream else None, ctypes.byref(out)))
    return out


def mot_ctx_destroy(ctx):
    lib().mot_ctx_destroy(ctx)


def mot_problem_create(ctx, n, h: float, eps_r, alpha: float, opt: mot_options | None = None):
    n_arr = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    eps = np.ascontiguousarray(eps_r, dtype=np.float64)
    if eps.size != int(n[0]) * int(n[1]) * int(n[2]):
        raise MotError(MOT_EINVAL, "eps_r size does not match the grid")
    out = ctypes.c_void_p()
    _check(lib().mot_problem_create(ctx, n_arr, float(h), _ptr(eps), float(alpha),
                                    ctypes.byref(opt) if opt is not None else None, ctypes.byref(out)))
    return out


def mot_problem_info_get(prob) -> mot_problem_info:
    info = mot_problem_info()
    _check(lib().mot_problem_info_get(prob, ctypes.byref(info)))
    return info


def mot_problem_schedule(prob, nrhs: int, dtype: int) -> dict:
    """The autotuned launch schedule of the Z0 product for (nrhs, dtype), as a dict."""
    sc = mot_schedule()
    _check(lib().mot_problem_schedule(prob, int(nrhs), int(dtype), ctypes.byref(sc)))
    return {f: getattr(sc, f) for f, _ in mot_schedule._fields_}


def mot_problem_destroy(prob):
    lib().mot_problem_destroy(prob)


def mot_apply_Z0(prob, x_dev, y_dev, nrhs: int, dtype: int):
    _check(lib().mot_apply_Z0(prob, _ptr(x_dev), _ptr(y_dev), int(nrhs), int(dtype)))


def mot_apply_Z0_static(prob, x_dev, y_dev, nrhs: int, dtype: int):
    """y = Z0 x using the library's static device scratch (no allocation)."""
    _check(lib().mot_apply_Z0_static(prob, _ptr(x_dev), _ptr(y_dev), int(nrhs), int(dtype)))


def mot_apply_Z0_direct(prob, x_dev, y_dev, nrhs: int, dtype: int):
    """y = Z0 x by direct summation over the lag-0 support (the paper's direct product)."""
    _check(lib().mot_apply_Z0_direct(prob, _ptr(x_dev), _ptr(y_dev), int(nrhs), int(dtype)))


def mot_kernel_table(prob, lag: int):
    R = (ctypes.c_int32 * 3)()
    _check(lib().mot_kernel_table(prob, int(lag), None, R))
    Rx, Ry, Rz = R[0], R[1], R[2]
    g = np.zeros((6, 2 * Rz + 1, 2 * Ry + 1, 2 * Rx + 1))
    _check(lib().mot_kernel_table(prob, int(lag), _ptr(g), R))
    return (Rx, Ry, Rz), g


def mot_set_kernel_table(prob, lag: int, g, R):
    g = np.ascontiguousarray(g, dtype=np.float64)
    Ra = (ctypes.c_int32 * 3)(*[int(v) for v in R])
    _check(lib().mot_set_kernel_table(prob, int(lag), _ptr(g), Ra))


def mot_table_host(rho: float, lag: int, R):
    Rx, Ry, Rz = (int(v) for v in R)
    g = np.zeros((6, 2 * Rz + 1, 2 * Ry + 1, 2 * Rx + 1))
    Ra = (ctypes.c_int32 * 3)(Rx, Ry, Rz)
    _check(lib().mot_table_host(float(rho), int(lag), Ra, _ptr(g)))
    return g


def _planewaves(exc):
    arr = (mot_planewave * len(exc))()
    for i, w in enumerate(exc):
        if isinstance(w, dict):
            arr[i].E0, arr[i].sigma, arr[i].t0, arr[i].f0 = w["E0"], w["sigma"], w["t0"], w["f0"]
            for j in range(3):
                arr[i].khat[j] = w["khat"][j]
                arr[i].pol[j] = w["pol"][j]
        else:
            arr[i] = w
    return arr


def mot_run_create(prob, exc, precision: int = MOT_FP64):
    arr = _planewaves(exc)
    out = ctypes.c_void_p()
    _check(lib().mot_run_create(prob, len(exc), arr, int(precision), ctypes.byref(out)))
    return out


def mot_run_step(run, nsteps: int, J_out=None, stats=None, allow_notconv: bool = False):
    if stats is not None and len(stats) < nsteps:
        raise ValueError(f"stats holds {len(stats)} entries, {nsteps} steps requested")
    st = lib().mot_run_step(run, int(nsteps), _ptr(J_out), ctypes.byref(stats[0]) if stats is not None else None)
    if st == MOT_ENOTCONV and allow_notconv:
        return st
    _check(st)
    return st


def mot_run_current_device(run) -> int:
    p = ctypes.c_void_p()
    _check(lib().mot_run_current_device(run, ctypes.byref(p)))
    return p.value


def mot_run_step_index(run) -> int:
    n = ctypes.c_int64()
    _check(lib().mot_run_step_index(run, ctypes.byref(n)))
    return n.value


def mot_run_save(run, path):
    """Write the run's state (J history, history ring, step index) to path."""
    _check(lib().mot_run_save(run, os.fsencode(path)))


def mot_run_load(prob, path):
    """A run resumed on prob from a checkpoint written by mot_run_save."""
    out = ctypes.c_void_p()
    _check(lib().mot_run_load(prob, os.fsencode(path), ctypes.byref(out)))
    return out


_served = {}  # (server, ticket) -> the host output array the library writes before the wait returns


def mot_server_create(ctx, mem_budget: int = 0, max_slots: int = 4):
    out = ctypes.c_void_p()
    _check(lib().mot_server_create(ctx, int(mem_budget), int(max_slots), ctypes.byref(out)))
    return out


def mot_server_submit(server, N, h, eps_r, alpha, exc, nsteps, precision=MOT_MIXED, opt=None, J_final=None) -> int:
    """Queue a run; J_final (C-contiguous float64 [nrhs, 3, nv] or None) receives the last step's J."""
    eps = np.ascontiguousarray(eps_r, dtype=np.float64)
    arr = _planewaves(exc)
    if J_final is not None:
        assert J_final.dtype == np.float64 and J_final.flags["C_CONTIGUOUS"]
        assert J_final.size == len(exc) * 3 * int(np.prod(N))
    q = mot_request()
    for i in range(3):
        q.n[i] = int(N[i])
    q.h, q.alpha, q.precision, q.nrhs, q.nsteps = float(h), float(alpha), int(precision), len(exc), int(nsteps)
    q.eps_r = eps.ctypes.data
    q.exc = ctypes.cast(arr, ctypes.c_void_p).value
    q.opt = ctypes.cast(ctypes.byref(opt), ctypes.c_void_p).value if opt is not None else None
    q.J_final = J_final.ctypes.data if J_final is not None else None
    t = ctypes.c_uint64()
    _check(lib().mot_server_submit(server, ctypes.byref(q), ctypes.byref(t)))
    _served[(server.value, t.value)] = J_final
    return t.value


def mot_server_wait(server, ticket: int, timeout_s: float = 60.0) -> mot_result:
    res = mot_result()
    _check(lib().mot_server_wait(server, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(res)))
    _served.pop((server.value, ticket), None)
    return res


def mot_server_destroy(server):
    lib().mot_server_destroy(server)
    for k in [k for k in _served if k[0] == server.value]:
        del _served[k]


def mot_run_kernel_times(run) -> dict:
    """{class name: (launches, mean ms)} of the latest step (timing option)."""
    out = {}
    for i, name in enumerate(KERNEL_CLASSES):
        n, ms = ctypes.c_int32(), ctypes.c_float()
        _check(lib().mot_run_kernel_times(run, i, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (n.value, ms.value)
    return out


def mot_kernel_launches() -> int:
    c = ctypes.c_uint64()
    _check(lib().mot_kernel_launches(ctypes.byref(c)))
    return c.value


def mot_fma_peak(device: int = 0, dtype: int = MOT_F64):
    """(FLOP/s, ms) of the library's FMA microkernel on `device`."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().mot_fma_peak(int(device), int(dtype), ctypes.byref(f), ctypes.byref(ms)))
    return f.value, ms.value


def default_options(**kw) -> mot_options:
    """mot_options with the library defaults (tol 0 = per-precision default)."""
    o = mot_options(0.0, 500, 1e-6, 6, 0.0, 0, 2, 1, 1)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def mot_run_destroy(run):
    lib().mot_run_destroy(run)
