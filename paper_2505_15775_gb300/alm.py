"""Python binding of the C ABI in ``include/alm.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Device arrays are
torch CUDA tensors; each handle runs on its own CUDA stream, ordered against
torch's current stream around every call.  There is no CPU path: if the shared
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libalm_gb300.so")

ALM_OK, ALM_ERR_INVALID_ARG, ALM_ERR_CUDA, ALM_ERR_OOM = 0, 1, 2, 3
ALM_ERR_NUMERIC, ALM_ERR_NOT_CONVERGED, ALM_ERR_TIMEOUT, ALM_ERR_UNBOUNDED = 4, 5, 6, 7
ALM_FP64, ALM_FP32 = 0, 1
ALM_INNER_CG, ALM_INNER_GD = 0, 1
ALM_SIGMA_FIXED, ALM_SIGMA_ADAPTIVE = 0, 1
STATUS_NAMES = {0: "ALM_OK", 1: "ALM_ERR_INVALID_ARG", 2: "ALM_ERR_CUDA", 3: "ALM_ERR_OOM",
                4: "ALM_ERR_NUMERIC", 5: "ALM_ERR_NOT_CONVERGED", 6: "ALM_ERR_TIMEOUT",
                7: "ALM_ERR_UNBOUNDED"}

EXPORTED = ["alm_default_options", "alm_create", "alm_destroy", "alm_last_error", "alm_pattern_info",
            "alm_eval", "alm_grad", "alm_linesearch", "alm_lambda_min", "alm_solve", "alm_version",
            "alm_checkpoint", "alm_resume", "alm_set_log", "alm_set_inner_shape", "alm_get_inner_shape", "alm_inner_shapes",
            "alm_autotune", "alm_cg_step",
            "alm_grad_unitdiag_noalloc", "alm_batch_create", "alm_batch_destroy", "alm_batch_last_error",
            "alm_batch_solve", "alm_batch_autotune", "alm_batch_set_threads", "alm_gnn_num_params",
            "alm_gnn_create", "alm_gnn_destroy", "alm_gnn_last_error", "alm_gnn_set_params", "alm_gnn_get_params",
            "alm_gnn_forward", "alm_gnn_warm_start", "alm_gnn_loss_grad", "alm_gnn_train"]
ALM_GNN_FP32, ALM_GNN_BF16 = 0, 1
ALM_BATCH_LDR = 32


class alm_problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64),
                ("c_nnz", C.c_int64), ("c_i", C.c_void_p), ("c_j", C.c_void_p), ("c_v", C.c_void_p),
                ("c_lr_k", C.c_int32), ("c_lr_u", C.c_void_p), ("c_lr_s", C.c_void_p),
                ("a_nnz", C.c_int64), ("a_k", C.c_void_p), ("a_i", C.c_void_p), ("a_j", C.c_void_p),
                ("a_v", C.c_void_p), ("b", C.c_void_p)]


class alm_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("r_max", C.c_int32), ("sigma0", C.c_double),
                ("sigma_rule", C.c_int32), ("sigma_max", C.c_double), ("eps", C.c_double),
                ("max_outer", C.c_int32), ("max_inner", C.c_int32), ("inner_method", C.c_int32),
                ("inner_rel", C.c_double), ("inner_floor", C.c_double), ("inner_start", C.c_double),
                ("inner_decay", C.c_double), ("lanczos_k", C.c_int32), ("lanczos_max_restarts", C.c_int32),
                ("lanczos_tol", C.c_double), ("seed", C.c_uint64), ("chunk", C.c_int32),
                ("use_graph", C.c_int32), ("profile", C.c_int32), ("verbose", C.c_int32),
                ("inner_precond", C.c_int32), ("lanczos_warm", C.c_int32), ("fallback_inner", C.c_int32),
                ("growth_k", C.c_int32)]


class alm_inner_shape(C.Structure):
    _fields_ = [("variant", C.c_int32), ("stages", C.c_int32), ("threads", C.c_int32)]


class alm_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer", C.c_int32), ("inner_total", C.c_int32), ("rank", C.c_int32),
                ("sigma", C.c_double), ("kkt", C.c_double * 3), ("objective", C.c_double),
                ("lambda_min", C.c_double), ("lanczos_matvecs", C.c_int64), ("kernel_launches", C.c_int64),
                ("spmm_launches", C.c_int64), ("spmm_ms", C.c_double), ("spmm_bytes", C.c_double),
                ("spmm_rank_pad", C.c_int32), ("growth_steps", C.c_int32), ("time_ms", C.c_double),
                ("step_ms", C.c_double * 5), ("lanczos_ms", C.c_double), ("ls_bytes", C.c_double)]


class alm_batch_problem(C.Structure):
    _fields_ = [("count", C.c_int32), ("row_off", C.c_void_p), ("nnz_off", C.c_void_p),
                ("c_i", C.c_void_p), ("c_j", C.c_void_p), ("c_v", C.c_void_p)]


class alm_instance_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer", C.c_int32), ("inner_total", C.c_int32), ("rank", C.c_int32),
                ("lanczos_matvecs", C.c_int32), ("growth_steps", C.c_int32), ("kkt", C.c_double * 3),
                ("objective", C.c_double), ("lambda_min", C.c_double), ("sigma", C.c_double),
                ("device_ms", C.c_double), ("fell_back", C.c_int32), ("reserved", C.c_int32)]


class alm_batch_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("converged", C.c_int32), ("threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("grid", C.c_int32), ("kernel_launches", C.c_int64),
                ("inner_total", C.c_int64), ("lanczos_matvecs", C.c_int64), ("device_ms", C.c_double),
                ("time_ms", C.c_double)]


_lib = None


def load() -> C.CDLL:
    """Load the CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run `python -m paper_2505_15775_gb300.build`)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    pd = C.POINTER(C.c_double)
    lib.alm_default_options.argtypes = [C.POINTER(alm_options)]
    lib.alm_default_options.restype = None
    lib.alm_create.argtypes = [C.POINTER(vp), C.POINTER(alm_problem), C.POINTER(alm_options), vp]
    lib.alm_create.restype = C.c_int
    lib.alm_destroy.argtypes = [vp]
    lib.alm_destroy.restype = None
    lib.alm_last_error.argtypes = [vp]
    lib.alm_last_error.restype = C.c_char_p
    lib.alm_pattern_info.argtypes = [vp, C.POINTER(C.c_int64)]
    lib.alm_pattern_info.restype = C.c_int
    lib.alm_eval.argtypes = [vp, vp, i32, i32, vp, dbl, pd, vp, pd]
    lib.alm_eval.restype = C.c_int
    lib.alm_grad.argtypes = [vp, vp, i32, i32, vp, dbl, vp, pd]
    lib.alm_grad.restype = C.c_int
    lib.alm_linesearch.argtypes = [vp, vp, vp, i32, i32, vp, dbl, pd, pd]
    lib.alm_linesearch.restype = C.c_int
    lib.alm_lambda_min.argtypes = [vp, vp, i32, i32, vp, dbl, pd, vp, pd]
    lib.alm_lambda_min.restype = C.c_int
    lib.alm_solve.argtypes = [vp, vp, i32, C.POINTER(C.c_int32), vp, C.POINTER(alm_stats)]
    lib.alm_solve.restype = C.c_int
    lib.alm_checkpoint.argtypes = [vp, C.c_char_p]
    lib.alm_checkpoint.restype = C.c_int
    lib.alm_set_log.argtypes = [vp, C.c_char_p]
    lib.alm_set_log.restype = C.c_int
    lib.alm_resume.argtypes = [vp, C.c_char_p, vp, i32, C.POINTER(C.c_int32), vp, C.POINTER(alm_stats)]
    lib.alm_resume.restype = C.c_int
    lib.alm_set_inner_shape.argtypes = [vp, C.POINTER(alm_inner_shape)]
    lib.alm_set_inner_shape.restype = C.c_int
    lib.alm_get_inner_shape.argtypes = [vp, C.POINTER(alm_inner_shape)]
    lib.alm_get_inner_shape.restype = C.c_int
    lib.alm_inner_shapes.argtypes = [C.POINTER(alm_inner_shape)]
    lib.alm_inner_shapes.restype = i32
    lib.alm_autotune.argtypes = [vp, vp, i32, i32, vp, i32, C.c_char_p, C.POINTER(alm_inner_shape), pd,
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.alm_autotune.restype = C.c_int
    lib.alm_cg_step.argtypes = [vp, vp, vp, i32, i32, vp, dbl, dbl, dbl, vp, vp, vp, vp, pd]
    lib.alm_cg_step.restype = C.c_int
    lib.alm_version.argtypes = []
    lib.alm_version.restype = C.c_char_p
    lib.alm_grad_unitdiag_noalloc.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, dbl, vp, i32, i32, vp, vp]
    lib.alm_grad_unitdiag_noalloc.restype = C.c_int
    lib.alm_batch_create.argtypes = [C.POINTER(vp), C.POINTER(alm_batch_problem), C.POINTER(alm_options), vp]
    lib.alm_batch_create.restype = C.c_int
    lib.alm_batch_destroy.argtypes = [vp]
    lib.alm_batch_destroy.restype = None
    lib.alm_batch_last_error.argtypes = [vp]
    lib.alm_batch_last_error.restype = C.c_char_p
    lib.alm_batch_solve.argtypes = [vp, vp, vp, vp, C.POINTER(alm_batch_stats), C.POINTER(alm_instance_stats)]
    lib.alm_batch_solve.restype = C.c_int
    lib.alm_batch_autotune.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int32), pd]
    lib.alm_batch_autotune.restype = C.c_int
    lib.alm_batch_set_threads.argtypes = [vp, i32]
    lib.alm_batch_set_threads.restype = C.c_int
    u64 = C.c_uint64
    lib.alm_gnn_num_params.argtypes = []
    lib.alm_gnn_num_params.restype = i32
    lib.alm_gnn_create.argtypes = [C.POINTER(vp), i32, u64, u64, vp]
    lib.alm_gnn_create.restype = C.c_int
    lib.alm_gnn_destroy.argtypes = [vp]
    lib.alm_gnn_destroy.restype = None
    lib.alm_gnn_last_error.argtypes = [vp]
    lib.alm_gnn_last_error.restype = C.c_char_p
    lib.alm_gnn_set_params.argtypes = [vp, vp]
    lib.alm_gnn_set_params.restype = C.c_int
    lib.alm_gnn_get_params.argtypes = [vp, vp]
    lib.alm_gnn_get_params.restype = C.c_int
    lib.alm_gnn_forward.argtypes = [vp, vp, vp, vp]
    lib.alm_gnn_forward.restype = C.c_int
    lib.alm_gnn_warm_start.argtypes = [vp, vp, dbl, vp, vp, vp]
    lib.alm_gnn_warm_start.restype = C.c_int
    lib.alm_gnn_loss_grad.argtypes = [vp, vp, vp, vp, dbl, pd, vp]
    lib.alm_gnn_loss_grad.restype = C.c_int
    lib.alm_gnn_train.argtypes = [vp, vp, vp, vp, dbl, i32, dbl, pd]
    lib.alm_gnn_train.restype = C.c_int
    _lib = lib
    return lib


class AlmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, h=None):
    if status != ALM_OK:
        msg = load().alm_last_error(h.ptr if h is not None else None)
        raise AlmError(status, (msg or b"").decode())


def default_options(**kw) -> alm_options:
    o = alm_options()
    load().alm_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class Handle:
    ptr: C.c_void_p
    n: int
    m: int
    precision: int
    dtype: torch.dtype
    options: alm_options
    stream: torch.cuda.Stream

    @property
    def width(self) -> int:          # elements per 16 bytes
        return 2 if self.precision == ALM_FP64 else 4

    def ldr_for(self, r: int) -> int:
        w = self.width
        return (r + w - 1) // w * w


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def _call(h: Handle, fn, *args) -> int:
    """Run one C call on the handle's stream, ordered after the work already queued
    on torch's current stream and before the work queued on it afterwards."""
    cur = torch.cuda.current_stream()
    h.stream.wait_stream(cur)
    st = fn(*args)
    cur.wait_stream(h.stream)
    return st


def alm_create(inst, stream: torch.cuda.Stream | None = None, **options) -> Handle:
    """alm_create from an ``sdp_instances.Instance`` (host arrays).  The handle runs on
    its own stream (a new one unless given): CUDA graph capture needs a stream other
    than the legacy default stream."""
    lib = load()
    o = default_options(**options)
    keep = dict(
        c_i=np.ascontiguousarray(inst.c_i, np.int32), c_j=np.ascontiguousarray(inst.c_j, np.int32),
        c_v=np.ascontiguousarray(inst.c_v, np.float64), a_k=np.ascontiguousarray(inst.a_k, np.int32),
        a_i=np.ascontiguousarray(inst.a_i, np.int32), a_j=np.ascontiguousarray(inst.a_j, np.int32),
        a_v=np.ascontiguousarray(inst.a_v, np.float64), b=np.ascontiguousarray(inst.b, np.float64),
        lr_u=np.ascontiguousarray(inst.c_lr_u, np.float64).reshape(-1),
        lr_s=np.ascontiguousarray(inst.c_lr_s, np.float64).reshape(-1))
    p = alm_problem(n=inst.n, m=inst.m, c_nnz=keep["c_i"].size, c_i=_p(keep["c_i"]), c_j=_p(keep["c_j"]),
                    c_v=_p(keep["c_v"]), c_lr_k=keep["lr_s"].size, c_lr_u=_p(keep["lr_u"]),
                    c_lr_s=_p(keep["lr_s"]), a_nnz=keep["a_k"].size, a_k=_p(keep["a_k"]),
                    a_i=_p(keep["a_i"]), a_j=_p(keep["a_j"]), a_v=_p(keep["a_v"]), b=_p(keep["b"]))
    stream = stream or torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    h = C.c_void_p()
    _check(lib.alm_create(C.byref(h), C.byref(p), C.byref(o), C.c_void_p(stream.cuda_stream)))
    dt = torch.float64 if o.precision == ALM_FP64 else torch.float32
    return Handle(ptr=h, n=inst.n, m=inst.m, precision=o.precision, dtype=dt, options=o, stream=stream)


def alm_destroy(h: Handle) -> None:
    if h is not None and h.ptr:
        _call(h, load().alm_destroy, h.ptr)
        h.ptr = C.c_void_p()


def alm_pattern_info(h: Handle) -> dict:
    out = (C.c_int64 * 7)()
    _check(load().alm_pattern_info(h.ptr, out), h)
    keys = ["n", "m", "nnz_upper", "nnz_full", "n_selector", "m_general", "off_dynamic"]
    return dict(zip(keys, list(out)))


def alm_version() -> str:
    return load().alm_version().decode()


def factor_tensor(h: Handle, R: np.ndarray | torch.Tensor, ldr: int | None = None) -> torch.Tensor:
    """Device factor in the ABI layout: n x ldr (ldr * element size % 16 == 0), zero padding."""
    R = torch.as_tensor(R)
    n, r = R.shape
    ldr = ldr or h.ldr_for(r)
    out = torch.zeros((n, ldr), dtype=h.dtype, device="cuda")
    out[:, :r] = R.to(device="cuda", dtype=h.dtype)
    return out


def _dev_y(h: Handle, y):
    if y is None:
        return None
    y = torch.as_tensor(y)
    return y.to(device="cuda", dtype=torch.float64).contiguous()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def alm_eval(h: Handle, R: torch.Tensor, r: int, y, sigma: float, want_ax: bool = True):
    """-> (L, A(RR^T) as a device tensor or None, <C, RR^T>)"""
    y = _dev_y(h, y)
    AX = torch.empty(h.m, dtype=torch.float64, device="cuda") if want_ax else None
    L, CX = C.c_double(), C.c_double()
    _check(_call(h, load().alm_eval, h.ptr, _ptr(R), r, R.shape[1], _ptr(y), float(sigma), C.byref(L), _ptr(AX),
                 C.byref(CX)), h)
    return L.value, AX, CX.value


def alm_grad(h: Handle, R: torch.Tensor, r: int, y, sigma: float):
    """-> (G = 2 S R in R's layout, ||G||_F^2)"""
    y = _dev_y(h, y)
    G = torch.empty_like(R)
    g2 = C.c_double()
    _check(_call(h, load().alm_grad, h.ptr, _ptr(R), r, R.shape[1], _ptr(y), float(sigma), _ptr(G), C.byref(g2)), h)
    return G, g2.value


def alm_linesearch(h: Handle, R: torch.Tensor, D: torch.Tensor, r: int, y, sigma: float):
    """-> (q0..q4 as a numpy array, alpha*)"""
    y = _dev_y(h, y)
    q = (C.c_double * 5)()
    a = C.c_double()
    _check(_call(h, load().alm_linesearch, h.ptr, _ptr(R), _ptr(D), r, R.shape[1], _ptr(y), float(sigma), q,
                 C.byref(a)), h)
    return np.array(list(q)), a.value


def alm_lambda_min(h: Handle, R: torch.Tensor | None, r: int, y, sigma: float):
    """-> (lambda, unit Ritz vector (device tensor), residual ||S v - lambda v||)"""
    y = _dev_y(h, y)
    v = torch.empty(h.n, dtype=h.dtype, device="cuda")
    lam, res = C.c_double(), C.c_double()
    ldr = R.shape[1] if R is not None else 0
    _check(_call(h, load().alm_lambda_min, h.ptr, _ptr(R), r if R is not None else 0, ldr, _ptr(y), float(sigma),
                 C.byref(lam), _ptr(v), C.byref(res)), h)
    return lam.value, v, res.value


def alm_solve(h: Handle, R0, y0=None, raise_on_not_converged: bool = False):
    """-> (R (n x r device tensor view), r, y (device), stats dict)"""
    R0 = torch.as_tensor(R0)
    n, r0 = R0.shape
    ldr = h.ldr_for(max(h.options.r_max, r0))
    R = factor_tensor(h, R0, ldr)
    y = torch.zeros(h.m, dtype=torch.float64, device="cuda") if y0 is None else _dev_y(h, y0).clone()
    r = C.c_int32(r0)
    st = alm_stats()
    status = _call(h, load().alm_solve, h.ptr, _ptr(R), ldr, C.byref(r), _ptr(y), C.byref(st))
    if status != ALM_OK and (status != ALM_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(status, h)
    stats = {k: getattr(st, k) for k, _ in alm_stats._fields_}
    stats["kkt"] = list(st.kkt)
    stats["step_ms"] = list(st.step_ms)
    return R[:, : r.value], r.value, y, stats


def _stats_dict(st: alm_stats) -> dict:
    d = {k: getattr(st, k) for k, _ in alm_stats._fields_}
    d["kkt"] = list(st.kkt)
    d["step_ms"] = list(st.step_ms)
    return d


def alm_checkpoint(h: Handle, path: str) -> None:
    """Save the state at the end of the last solve on h (see include/alm.h)."""
    _check(_call(h, load().alm_checkpoint, h.ptr, os.fsencode(path)), h)


def alm_set_log(h: Handle, path: str | None) -> None:
    """Append one JSON line per outer iteration of every later solve on h to `path`
    (None switches it off; see include/alm.h for the fields)."""
    _check(load().alm_set_log(h.ptr, os.fsencode(path) if path else None), h)


def alm_resume(h: Handle, path: str, raise_on_not_converged: bool = False):
    """Continue a saved trajectory; -> (R (n x r device view), r, y (device), stats dict)"""
    ldr = h.ldr_for(h.options.r_max)
    R = torch.zeros((h.n, ldr), dtype=h.dtype, device="cuda")
    y = torch.zeros(h.m, dtype=torch.float64, device="cuda")
    r = C.c_int32(0)
    st = alm_stats()
    status = _call(h, load().alm_resume, h.ptr, os.fsencode(path), _ptr(R), ldr, C.byref(r), _ptr(y), C.byref(st))
    if status != ALM_OK and (status != ALM_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(status, h)
    return R[:, : r.value], r.value, y, _stats_dict(st)


def _shape_dict(s: alm_inner_shape) -> dict:
    return {"variant": s.variant, "stages": s.stages, "threads": s.threads}


def alm_set_inner_shape(h: Handle, variant: int, stages: int = 2, threads: int = 128):
    s = alm_inner_shape(variant, stages, threads)
    _check(load().alm_set_inner_shape(h.ptr, C.byref(s)), h)


def alm_get_inner_shape(h: Handle) -> dict:
    s = alm_inner_shape()
    _check(load().alm_get_inner_shape(h.ptr, C.byref(s)), h)
    return _shape_dict(s)


def alm_inner_shapes() -> list[dict]:
    buf = (alm_inner_shape * 16)()
    n = load().alm_inner_shapes(buf)
    return [_shape_dict(buf[k]) for k in range(n)]


def alm_autotune(h: Handle, R: torch.Tensor, r: int, y=None, steps: int = 16, cache: str | None = None):
    """Time the candidate launch shapes of the inner-step kernels on (R, y) and keep the
    fastest on h, or take it from the JSON-lines cache file `cache` when it holds this
    problem's key.  -> (chosen shape, [(shape, ms of `steps` inner steps)], from_cache)."""
    y = _dev_y(h, y if y is not None else np.zeros(h.m))
    best = alm_inner_shape()
    times = (C.c_double * 16)()
    cnt = C.c_int32(0)
    hit = C.c_int32(0)
    _check(_call(h, load().alm_autotune, h.ptr, _ptr(R), int(r), R.shape[1], _ptr(y), int(steps),
                 os.fsencode(cache) if cache else None, C.byref(best), times, C.byref(cnt), C.byref(hit)), h)
    shapes = alm_inner_shapes()
    return _shape_dict(best), [(shapes[k], times[k]) for k in range(cnt.value)], bool(hit.value)


def alm_cg_step(h: Handle, R: torch.Tensor, D: torch.Tensor, Zold: torch.Tensor, r: int, y, sigma: float,
                alpha: float, zg_prev: float):
    """One inner step of the fused inner loop from the state (R, D, Z_old, y, alpha, zg_prev).
    -> (R_out, Z, D_new, diag(S) (device), dict of gg, go, gd, zg, beta, q (q[0] not
    computed), alpha)"""
    y = _dev_y(h, y)
    Ro, Dn = torch.empty_like(R), torch.empty_like(R)
    Z = Zold.clone()
    diag = torch.empty(h.n, dtype=torch.float64, device="cuda")
    out = (C.c_double * 11)()
    _check(_call(h, load().alm_cg_step, h.ptr, _ptr(R), _ptr(D), int(r), R.shape[1], _ptr(y), float(sigma),
                 float(alpha), float(zg_prev), _ptr(Ro), _ptr(Z), _ptr(Dn), _ptr(diag), out), h)
    o = list(out)
    return Ro, Z, Dn, diag, {"gg": o[0], "go": o[1], "gd": o[2], "zg": o[3], "beta": o[4],
                             "q": np.array(o[5:10]), "alpha": o[10]}


def alm_grad_unitdiag_noalloc(precision: int, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                              cdiag: torch.Tensor, b: torch.Tensor, y: torch.Tensor, sigma: float,
                              R: torch.Tensor, r: int, G: torch.Tensor,
                              stream: torch.cuda.Stream | None = None) -> None:
    """G = 2 S R for problems with constraints X_ii = b_i, from caller-owned device tensors,
    with no device allocation inside the library (see include/alm.h).  Runs on `stream`
    (default: torch's current stream) and does not synchronise."""
    stream = stream or torch.cuda.current_stream()
    n = rowptr.numel() - 1
    _check(load().alm_grad_unitdiag_noalloc(precision, n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(cdiag), _ptr(b),
                                            _ptr(y), float(sigma), _ptr(R), r, R.shape[1], _ptr(G),
                                            C.c_void_p(stream.cuda_stream)))


# ------------------------------------------------------------------------------------
# batched solver (alm_batch_*)
# ------------------------------------------------------------------------------------
@dataclass
class BatchHandle:
    ptr: C.c_void_p
    count: int
    row_off: np.ndarray
    options: alm_options
    stream: torch.cuda.Stream

    @property
    def rows(self) -> int:
        return int(self.row_off[-1])


def _check_batch(status: int, hb=None):
    if status != ALM_OK:
        msg = load().alm_batch_last_error(hb.ptr if hb is not None else None)
        raise AlmError(status, (msg or b"").decode())


def batch_pack(instances) -> dict:
    """Concatenate the C data of unit-diagonal instances (``sdp_instances.Instance``) into
    the host arrays of ``alm_batch_problem`` (row and entry offsets, local COO)."""
    ns = np.array([inst.n for inst in instances], np.int64)
    nz = np.array([inst.c_i.size for inst in instances], np.int64)
    row_off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    nnz_off = np.concatenate([[0], np.cumsum(nz)]).astype(np.int64)
    cat = lambda key, dt: np.ascontiguousarray(np.concatenate([getattr(x, key) for x in instances]), dt)
    return dict(row_off=row_off, nnz_off=nnz_off, c_i=cat("c_i", np.int32), c_j=cat("c_j", np.int32),
                c_v=cat("c_v", np.float64))


def alm_batch_create(instances, stream: torch.cuda.Stream | None = None, **options) -> BatchHandle:
    """alm_batch_create from a list of unit-diagonal instances (precision ALM_FP32)."""
    lib = load()
    options.setdefault("precision", ALM_FP32)
    options.setdefault("lanczos_warm", 1)  # the batched solver's default (include/alm.h)
    o = default_options(**options)
    keep = batch_pack(instances)
    p = alm_batch_problem(count=len(instances), row_off=_p(keep["row_off"]), nnz_off=_p(keep["nnz_off"]),
                          c_i=_p(keep["c_i"]), c_j=_p(keep["c_j"]), c_v=_p(keep["c_v"]))
    stream = stream or torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    h = C.c_void_p()
    _check_batch(lib.alm_batch_create(C.byref(h), C.byref(p), C.byref(o), C.c_void_p(stream.cuda_stream)))
    return BatchHandle(ptr=h, count=len(instances), row_off=keep["row_off"], options=o, stream=stream)


def alm_batch_destroy(hb: BatchHandle) -> None:
    if hb is not None and hb.ptr:
        _call(hb, load().alm_batch_destroy, hb.ptr)
        hb.ptr = C.c_void_p()


def batch_factor(hb: BatchHandle, factors) -> tuple[torch.Tensor, torch.Tensor]:
    """Device (rows x 32) float factor and int32 ranks from per-instance n_b x r_b arrays."""
    R = torch.zeros((hb.rows, ALM_BATCH_LDR), dtype=torch.float32)
    ranks = np.zeros(hb.count, np.int32)
    for b, F in enumerate(factors):
        F = torch.as_tensor(np.asarray(F), dtype=torch.float32)
        R[int(hb.row_off[b]):int(hb.row_off[b + 1]), : F.shape[1]] = F
        ranks[b] = F.shape[1]
    return R.to("cuda"), torch.as_tensor(ranks, device="cuda")


def alm_batch_solve(hb: BatchHandle, R: torch.Tensor, rank: torch.Tensor, y: torch.Tensor,
                    raise_on_not_converged: bool = False):
    """Solve in place (R: rows x 32 float, rank: int32 per instance, y: float64 per row).
    -> (batch stats dict, per-instance list of stats dicts)"""
    st = alm_batch_stats()
    per = (alm_instance_stats * hb.count)()
    status = _call(hb, load().alm_batch_solve, hb.ptr, _ptr(R), _ptr(rank), _ptr(y), C.byref(st), per)
    if status != ALM_OK and (status not in (ALM_ERR_NOT_CONVERGED, ALM_ERR_NUMERIC, ALM_ERR_UNBOUNDED)
                             or raise_on_not_converged):
        _check_batch(status, hb)
    stats = {k: getattr(st, k) for k, _ in alm_batch_stats._fields_}
    inst = []
    for x in per:
        d = {k: getattr(x, k) for k, _ in alm_instance_stats._fields_}
        d["kkt"] = list(x.kkt)
        inst.append(d)
    return stats, inst


def alm_batch_autotune(hb: BatchHandle, R: torch.Tensor, rank: torch.Tensor, y: torch.Tensor):
    """-> (chosen threads per CTA, {threads: sample time in ms})"""
    t = C.c_int32()
    times = (C.c_double * 3)()
    _check_batch(_call(hb, load().alm_batch_autotune, hb.ptr, _ptr(R), _ptr(rank), _ptr(y), C.byref(t), times), hb)
    return t.value, dict(zip((256, 512, 1024), list(times)))


def alm_batch_set_threads(hb: BatchHandle, threads: int) -> None:
    _check_batch(load().alm_batch_set_threads(hb.ptr, int(threads)), hb)


# ------------------------------------------------------------------------------------
# warm-start network (alm_gnn_*)
# ------------------------------------------------------------------------------------
@dataclass
class GnnHandle:
    ptr: C.c_void_p
    storage: int
    stream: torch.cuda.Stream


def _check_gnn(status: int, g=None):
    if status != ALM_OK:
        msg = load().alm_gnn_last_error(g.ptr if g is not None else None)
        raise AlmError(status, (msg or b"").decode())


def alm_gnn_num_params() -> int:
    return int(load().alm_gnn_num_params())


def alm_gnn_create(storage: int = ALM_GNN_BF16, feat_seed: int = 0x6E6E, init_seed: int = 1,
                   stream: torch.cuda.Stream | None = None) -> GnnHandle:
    stream = stream or torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    h = C.c_void_p()
    _check_gnn(load().alm_gnn_create(C.byref(h), int(storage), int(feat_seed), int(init_seed),
                                     C.c_void_p(stream.cuda_stream)))
    return GnnHandle(ptr=h, storage=int(storage), stream=stream)


def alm_gnn_destroy(g: GnnHandle) -> None:
    if g is not None and g.ptr:
        _call(g, load().alm_gnn_destroy, g.ptr)
        g.ptr = C.c_void_p()


def alm_gnn_set_params(g: GnnHandle, theta) -> None:
    th = np.ascontiguousarray(theta, np.float32)
    assert th.size == alm_gnn_num_params()
    _check_gnn(_call(g, load().alm_gnn_set_params, g.ptr, th.ctypes.data_as(C.c_void_p)), g)


def alm_gnn_get_params(g: GnnHandle) -> np.ndarray:
    th = np.zeros(alm_gnn_num_params(), np.float32)
    _check_gnn(_call(g, load().alm_gnn_get_params, g.ptr, th.ctypes.data_as(C.c_void_p)), g)
    return th


def alm_gnn_forward(g: GnnHandle, hb: BatchHandle):
    """-> (rhat rows x 32 float tensor, yhat rows float tensor)"""
    rhat = torch.empty((hb.rows, 32), dtype=torch.float32, device="cuda")
    yhat = torch.empty(hb.rows, dtype=torch.float32, device="cuda")
    _check_gnn(_call(g, load().alm_gnn_forward, g.ptr, hb.ptr, _ptr(rhat), _ptr(yhat)), g)
    return rhat, yhat


def alm_gnn_warm_start(g: GnnHandle, hb: BatchHandle, mix: float = 1.0):
    """-> (R0 rows x 32 float, rank int32 per instance, y0 float64 per row), device tensors"""
    R0 = torch.empty((hb.rows, ALM_BATCH_LDR), dtype=torch.float32, device="cuda")
    rank = torch.empty(hb.count, dtype=torch.int32, device="cuda")
    y0 = torch.empty(hb.rows, dtype=torch.float64, device="cuda")
    _check_gnn(_call(g, load().alm_gnn_warm_start, g.ptr, hb.ptr, float(mix), _ptr(R0), _ptr(rank), _ptr(y0)), g)
    return R0, rank, y0


def alm_gnn_loss_grad(g: GnnHandle, hb: BatchHandle, Rstar: torch.Tensor, ystar: torch.Tensor, lam: float):
    """-> (loss, gradient as a float32 numpy vector)"""
    loss = C.c_double()
    grad = np.zeros(alm_gnn_num_params(), np.float32)
    _check_gnn(_call(g, load().alm_gnn_loss_grad, g.ptr, hb.ptr, _ptr(Rstar), _ptr(ystar), float(lam),
                     C.byref(loss), grad.ctypes.data_as(C.c_void_p)), g)
    return loss.value, grad


def alm_gnn_train(g: GnnHandle, hb: BatchHandle, Rstar: torch.Tensor, ystar: torch.Tensor, lam: float,
                  steps: int, lr: float) -> np.ndarray:
    """`steps` Adam steps; -> the loss before each step"""
    losses = np.zeros(max(int(steps), 1), np.float64)
    _check_gnn(_call(g, load().alm_gnn_train, g.ptr, hb.ptr, _ptr(Rstar), _ptr(ystar), float(lam), int(steps),
                     float(lr), losses.ctypes.data_as(C.POINTER(C.c_double))), g)
    return losses[: int(steps)]
