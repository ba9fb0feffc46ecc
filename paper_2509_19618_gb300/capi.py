"""ctypes binding of libhpmxp.so (include/hpmxp.h, include/hpmxp_serve.h,
include/hpmxp_testing.h).

The ``hpmxp_*`` functions here have the C names and take raw pointers (ints),
sizes and a stream handle; they only marshal arguments.  PyTorch is used by
the friendlier wrappers in ``api.py`` for device memory and streams.  There is
no fallback: importing this module on a machine where the library cannot be
built or loaded raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ETIMEOUT, EINVALID = range(8)
BF16, FP16, FP8_E4M3, BF16_TRAIL32, FP16_TRAIL32 = 0, 1, 2, 3, 4
DIAG_DOMINANT, DIAG_SQRTN, DIAG_NONE, DIAG_DEPARTURE = 0, 1, 2, 3
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "EBREAKDOWN",
                6: "ETIMEOUT", 7: "EINVALID"}


class IRParams(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("theta", ctypes.c_double), ("accept", ctypes.c_double), ("precond_fp32", ctypes.c_int32),
                ("matvec_fp32", ctypes.c_int32)]


class IRInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("scaled_resid", ctypes.c_double),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("gemm_tile", ctypes.c_int32), ("reserve_sms", ctypes.c_int32), ("overlap_min", ctypes.c_int64),
                ("sm_budget", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("LU", ctypes.c_void_p),
                ("ldlu", ctypes.c_int64), ("b", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("x", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("nrhs", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("n", ctypes.c_int64), ("nrhs", ctypes.c_int64), ("prec", ctypes.c_int32),
                ("nb", ctypes.c_int32), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("b", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("x", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("margin", ctypes.c_double), ("diag_mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("params", IRParams)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("info", IRInfo * 8), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class HpmxpError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)} ({status_string(status)})")


def library_path() -> str:
    return _build.LIB


def load():
    """Load (building first if stale) libhpmxp.so and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _build.stale():
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        i64, u64, i32, d, sz, P = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_size_t, ctypes.c_void_p)
        sig = {
            "hpmxp_status_string": ([i32], ctypes.c_char_p),
            "hpmxp_version": ([], i32),
            "hpmxp_generate_workspace": ([i64], sz),
            "hpmxp_generate": ([i64, u64, d, i32, P, i64, P, i64, i64, P, sz, P], i32),
            "hpmxp_generate_noalloc": ([i64, u64, d, i32, P, i64, P, i64, i64, P], i32),
            "hpmxp_factor_workspace": ([i64, i32, i32], sz),
            "hpmxp_factor": ([i64, P, i64, i32, i32, P, i64, P, sz, P], i32),
            "hpmxp_factor_scaled": ([i64, P, i64, i32, i32, P, P, P, i64, P, sz, P], i32),
            "hpmxp_factor_batched_workspace": ([ctypes.POINTER(Problem), i32, i32], sz),
            "hpmxp_factor_batched": ([ctypes.POINTER(Problem), i32, i32, ctypes.POINTER(i32), P, sz, P], i32),
            "hpmxp_solve_ir_batched_workspace": ([ctypes.POINTER(Problem), i32, i32], sz),
            "hpmxp_solve_ir_batched": ([ctypes.POINTER(Problem), i32, i32, ctypes.POINTER(IRParams),
                                        ctypes.POINTER(IRInfo), P, sz, P], i32),
            "hpmxp_balance": ([i64, P, i64, i32, P, P, P], i32),
            "hpmxp_ir_params_default": ([ctypes.POINTER(IRParams)], None),
            "hpmxp_solve_workspace": ([i64, i64, i32], sz),
            "hpmxp_solve_workspace_a32": ([i64], sz),
            "hpmxp_solve_ir": ([i64, P, i64, P, i64, i32, P, i64, P, i64, i64, ctypes.POINTER(IRParams),
                                ctypes.POINTER(IRInfo), P, sz, P], i32),
            "hpmxp_solve_ir_scaled": ([i64, P, i64, P, i64, i32, P, P, P, i64, P, i64, i64,
                                       ctypes.POINTER(IRParams), ctypes.POINTER(IRInfo), P, sz, P], i32),
            "hpmxp_residual_workspace": ([i64, i64], sz),
            "hpmxp_residual": ([i64, P, i64, P, i64, P, i64, i64, P, P, sz, P], i32),
            "hpmxp_residual_vector": ([i64, P, i64, P, i64, P, i64, i64, P, i64, P, sz, P], i32),
            "hpmxp_lu_f64_workspace": ([i64], sz),
            "hpmxp_lu_f64": ([i64, P, i64, P, sz, P], i32),
            "hpmxp_lu_solve_f64": ([i64, P, i64, P, i64, i64, P], i32),
            "hpmxp_test_gemm": ([i32, i32, i32, P, i64, P, i64, P, i64, P, i64, i32, ctypes.c_float, i32, i32,
                                 P, i32, P, i32, i32, P, P], i32),
            "hpmxp_test_cast": ([i64, P, i64, i32, P, i64, P], i32),
            "hpmxp_launch_count": ([], ctypes.c_ulonglong),
            "hpmxp_set_tuning": ([ctypes.POINTER(Tuning)], i32),
            "hpmxp_get_tuning": ([ctypes.POINTER(Tuning)], None),
            "hpmxp_prof_enable": ([i32], None),
            "hpmxp_prof_read_device": ([i32, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)], i32),
            "hpmxp_prof_reset": ([], None),
            "hpmxp_prof_read": ([i32, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)], i32),
            "hpmxp_prof_read_bytes": ([i32, ctypes.POINTER(d)], i32),
            "hpmxp_prof_timeline": ([P, i32], i32),
            "hpmxp_test_precond": ([i64, P, i64, i32, P, i64, P, i64, i64, i32, P, sz, P], i32),
            "hpmxp_test_arena": ([sz, ctypes.POINTER(i64), i32, ctypes.POINTER(i64)], i32),
            "hpmxp_test_fill_smem": ([ctypes.c_uint32, P], i32),
            "hpmxp_test_decode16": ([P, P, i64, i32, P], i32),
            "hpmxp_test_set_wait_budget": ([ctypes.c_longlong, ctypes.c_ulonglong], i32),
            "hpmxp_request_footprint": ([ctypes.POINTER(Request)], sz),
            "hpmxp_executor_create": ([i32, i32, P, sz, ctypes.POINTER(P)], i32),
            "hpmxp_executor_create_batched": ([i32, i32, i32, P, sz, ctypes.POINTER(P)], i32),
            "hpmxp_executor_submit": ([P, ctypes.POINTER(Request)], i32),
            "hpmxp_executor_poll": ([P, ctypes.POINTER(Completion), i32, i32], i32),
            "hpmxp_executor_outstanding": ([P], i64),
            "hpmxp_executor_clock": ([P], d),
            "hpmxp_executor_destroy": ([P], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return load().hpmxp_status_string(s).decode()


def declared_symbols() -> list[str]:
    """Every function declared in include/*.h."""
    names = []
    inc = os.path.join(_build.ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            text = open(os.path.join(inc, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(hpmxp_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def _call(name: str, *args) -> int:
    return getattr(load(), name)(*args)


def hpmxp_generate_workspace(n):
    return _call("hpmxp_generate_workspace", n)


def hpmxp_generate(n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, ws, ws_bytes, stream):
    return _call("hpmxp_generate", n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, ws, ws_bytes, stream)


def hpmxp_generate_noalloc(n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, stream):
    return _call("hpmxp_generate_noalloc", n, seed, margin, diag_mode, A, lda, b, ldb, nrhs, stream)


def hpmxp_factor_workspace(n, prec, nb):
    return _call("hpmxp_factor_workspace", n, prec, nb)


def hpmxp_factor(n, A, lda, prec, nb, LU, ldlu, ws, ws_bytes, stream):
    return _call("hpmxp_factor", n, A, lda, prec, nb, LU, ldlu, ws, ws_bytes, stream)


def hpmxp_factor_scaled(n, A, lda, prec, nb, rs, cs, LU, ldlu, ws, ws_bytes, stream):
    return _call("hpmxp_factor_scaled", n, A, lda, prec, nb, rs, cs, LU, ldlu, ws, ws_bytes, stream)


def hpmxp_factor_batched_workspace(probs, prec):
    arr = (Problem * len(probs))(*probs)
    return _call("hpmxp_factor_batched_workspace", arr, len(probs), prec)


def hpmxp_factor_batched(probs, prec, ws, ws_bytes, stream):
    """Returns (status, [per-system status])."""
    arr = (Problem * len(probs))(*probs)
    per = (ctypes.c_int * len(probs))()
    st = _call("hpmxp_factor_batched", arr, len(probs), prec, per, ws, ws_bytes, stream)
    return st, list(per)


def hpmxp_solve_ir_batched_workspace(probs, restart):
    arr = (Problem * len(probs))(*probs)
    return _call("hpmxp_solve_ir_batched_workspace", arr, len(probs), restart)


def hpmxp_solve_ir_batched(probs, prec, params, info, ws, ws_bytes, stream):
    arr = (Problem * len(probs))(*probs)
    return _call("hpmxp_solve_ir_batched", arr, len(probs), prec, None if params is None else ctypes.byref(params),
                 info, ws, ws_bytes, stream)


def hpmxp_balance(n, A, lda, prec, rs, cs, stream):
    return _call("hpmxp_balance", n, A, lda, prec, rs, cs, stream)


def hpmxp_ir_params_default() -> IRParams:
    p = IRParams()
    load().hpmxp_ir_params_default(ctypes.byref(p))
    return p


def hpmxp_solve_workspace(n, nrhs, restart):
    return _call("hpmxp_solve_workspace", n, nrhs, restart)


def hpmxp_solve_ir(n, A, lda, LU, ldlu, prec, b, ldb, x, ldx, nrhs, params, info, ws, ws_bytes, stream):
    return _call("hpmxp_solve_ir", n, A, lda, LU, ldlu, prec, b, ldb, x, ldx, nrhs,
                 None if params is None else ctypes.byref(params), info, ws, ws_bytes, stream)


def hpmxp_solve_ir_scaled(n, A, lda, LU, ldlu, prec, rs, cs, b, ldb, x, ldx, nrhs, params, info, ws, ws_bytes,
                          stream):
    return _call("hpmxp_solve_ir_scaled", n, A, lda, LU, ldlu, prec, rs, cs, b, ldb, x, ldx, nrhs,
                 None if params is None else ctypes.byref(params), info, ws, ws_bytes, stream)


def hpmxp_solve_workspace_a32(n):
    return _call("hpmxp_solve_workspace_a32", n)


def hpmxp_residual_workspace(n, nrhs):
    return _call("hpmxp_residual_workspace", n, nrhs)


def hpmxp_residual(n, A, lda, x, ldx, b, ldb, nrhs, out, ws, ws_bytes, stream):
    return _call("hpmxp_residual", n, A, lda, x, ldx, b, ldb, nrhs, out, ws, ws_bytes, stream)


def hpmxp_residual_vector(n, A, lda, x, ldx, b, ldb, nrhs, r, ldr, ws, ws_bytes, stream):
    return _call("hpmxp_residual_vector", n, A, lda, x, ldx, b, ldb, nrhs, r, ldr, ws, ws_bytes, stream)


def hpmxp_lu_f64_workspace(n):
    return _call("hpmxp_lu_f64_workspace", n)


def hpmxp_lu_f64(n, A, lda, ws, ws_bytes, stream):
    return _call("hpmxp_lu_f64", n, A, lda, ws, ws_bytes, stream)


def hpmxp_lu_solve_f64(n, LU, ld, B, ldb, nrhs, stream):
    return _call("hpmxp_lu_solve_f64", n, LU, ld, B, ldb, nrhs, stream)


def hpmxp_set_tuning(gemm_tile: int = 0, reserve_sms: int = 0, overlap_min: int = 0, sm_budget: int = 0,
                     reserved: int = 0) -> int:
    t = Tuning(gemm_tile, reserve_sms, overlap_min, sm_budget, reserved)
    return load().hpmxp_set_tuning(ctypes.byref(t))


def hpmxp_get_tuning() -> dict:
    t = Tuning()
    load().hpmxp_get_tuning(ctypes.byref(t))
    return dict(gemm_tile=t.gemm_tile, reserve_sms=t.reserve_sms, overlap_min=t.overlap_min, sm_budget=t.sm_budget)


def hpmxp_launch_count() -> int:
    return int(load().hpmxp_launch_count())


def hpmxp_prof_enable(on: bool):
    load().hpmxp_prof_enable(1 if on else 0)


def hpmxp_prof_reset():
    load().hpmxp_prof_reset()


PROF_GEMM, PROF_GEMV, PROF_PRECOND, PROF_GETRF, PROF_GEMV32, PROF_CAST, PROF_PANEL, PROF_GEMM_STORE, \
    PROF_BALANCE = range(9)
PROF_NAMES = {0: "gemm_update", 1: "gemv", 2: "precond", 3: "getrf", 4: "gemv32", 5: "cast", 6: "panel",
              7: "gemm_panel", 8: "balance"}


def hpmxp_prof_read_device(kind: int) -> dict:
    """Execution time the kernels of a kind measured on the device (GEMM kinds)."""
    ms, cnt = ctypes.c_double(), ctypes.c_longlong()
    st = load().hpmxp_prof_read_device(kind, ctypes.byref(ms), ctypes.byref(cnt))
    if st != OK:
        raise HpmxpError("hpmxp_prof_read_device", st)
    return dict(ms=ms.value, launches=cnt.value)


def hpmxp_prof_read(kind: int) -> dict:
    ms, work, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    st = load().hpmxp_prof_read(kind, ctypes.byref(ms), ctypes.byref(work), ctypes.byref(cnt))
    if st != OK:
        raise HpmxpError("hpmxp_prof_read", st)
    by = ctypes.c_double()
    load().hpmxp_prof_read_bytes(kind, ctypes.byref(by))
    return dict(ms=ms.value, work=work.value, launches=cnt.value, bytes=by.value)


def hpmxp_test_gemm(*args):
    return _call("hpmxp_test_gemm", *args)


def hpmxp_test_cast(*args):
    return _call("hpmxp_test_cast", *args)


def hpmxp_test_precond(*args):
    return _call("hpmxp_test_precond", *args)


def hpmxp_test_fill_smem(pattern: int, stream) -> int:
    return _call("hpmxp_test_fill_smem", pattern, stream)


def hpmxp_test_decode16(codes, out, count: int, fmt: int, stream) -> int:
    return _call("hpmxp_test_decode16", codes, out, count, fmt, stream)


def hpmxp_test_set_wait_budget(polls: int, ns: int) -> int:
    return _call("hpmxp_test_set_wait_budget", polls, ns)


def hpmxp_test_arena(arena_bytes: int, ops: list[int]) -> list[int]:
    n = len(ops)
    a = (ctypes.c_int64 * max(n, 1))(*ops)
    r = (ctypes.c_int64 * max(n, 1))()
    st = load().hpmxp_test_arena(arena_bytes, a, n, r)
    if st != OK:
        raise HpmxpError("hpmxp_test_arena", st)
    return list(r[:n])


def hpmxp_request_footprint(req: Request) -> int:
    return int(load().hpmxp_request_footprint(ctypes.byref(req)))


def hpmxp_executor_create(device: int, workers: int, arena: int, arena_bytes: int):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().hpmxp_executor_create(device, workers, arena, arena_bytes, ctypes.byref(h))
    return st, h


def hpmxp_executor_create_batched(device: int, workers: int, max_batch: int, arena: int, arena_bytes: int):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().hpmxp_executor_create_batched(device, workers, max_batch, arena, arena_bytes, ctypes.byref(h))
    return st, h


def hpmxp_executor_submit(ex, req: Request) -> int:
    return _call("hpmxp_executor_submit", ex, ctypes.byref(req))


def hpmxp_executor_poll(ex, out, max_count: int, timeout_ms: int) -> int:
    return _call("hpmxp_executor_poll", ex, out, max_count, timeout_ms)


def hpmxp_executor_outstanding(ex) -> int:
    return int(_call("hpmxp_executor_outstanding", ex))


def hpmxp_executor_clock(ex) -> float:
    return float(_call("hpmxp_executor_clock", ex))


def hpmxp_executor_destroy(ex) -> int:
    return _call("hpmxp_executor_destroy", ex)


def hpmxp_prof_timeline() -> list[tuple[int, float, float]]:
    """Recorded spans since the last reset: (kind, start ms, end ms)."""
    n = int(load().hpmxp_prof_timeline(None, 0))
    buf = (ctypes.c_double * max(3 * n, 1))()
    n = min(n, int(load().hpmxp_prof_timeline(buf, n)))
    return [(int(buf[3 * i]), buf[3 * i + 1], buf[3 * i + 2]) for i in range(n)]
