"""CPU oracle for the HPL-MxP solver path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, sequential C++ (``hpmxp_oracle.cpp``) behind ctypes.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package; the solver library never does, and the oracle shares no
code with it.

Formats: 0 BF16, 1 FP16, 2 E4M3, 3 FP32, 4 FP64 (identity).
Diagonal modes: 0 DOMINANT (row absolute sum + margin), 1 SQRTN (margin sqrt(n)), 2 NONE,
3 DEPARTURE (margin times the row absolute sum).
Status codes returned by ``solve_ir``: 0 ok, 4 no convergence, 5 breakdown.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpmxp_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BF16, FP16, E4M3, FP32, FP64 = 0, 1, 2, 3, 4
DOMINANT, SQRTN, NONE, DEPARTURE = 0, 1, 2, 3


def _cpu_has_fma() -> bool:
    try:
        with open("/proc/cpuinfo") as f:
            return " fma " in f.read()
    except OSError:
        return False


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    flags = ["-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    if platform.machine() in ("x86_64", "AMD64") and _cpu_has_fma():
        flags.append("-mfma")  # explicit fmaf calls become single instructions; results unchanged
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", *flags, "-fopenmp", _SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        cmd.remove("-fopenmp")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB)
    return _LIB


class IRInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("scaled_resid", ctypes.c_double), ("status", ctypes.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i64, u64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
            P = ctypes.c_void_p
            L.oracle_round.argtypes = [d, i32]; L.oracle_round.restype = d
            L.oracle_round_array.argtypes = [P, P, i64, i32]; L.oracle_round_array.restype = None
            L.oracle_lcg_jump.argtypes = [u64, P, P]; L.oracle_lcg_jump.restype = None
            L.oracle_lcg_state.argtypes = [u64, u64]; L.oracle_lcg_state.restype = u64
            L.oracle_lcg_sequence.argtypes = [u64, i64, P]; L.oracle_lcg_sequence.restype = None
            L.oracle_draw_value.argtypes = [u64, u64]; L.oracle_draw_value.restype = d
            L.oracle_generate.argtypes = [i64, u64, d, i32, P, i64, P, i64, i64]
            L.oracle_generate.restype = i32
            L.oracle_generate_rows.argtypes = [i64, u64, d, i32, P, i64, P]
            L.oracle_generate_rows.restype = i32
            L.oracle_factor.argtypes = [i64, P, i64, i32, i32, i32, P, i64]
            L.oracle_factor.restype = i32
            L.oracle_factor_scheme.argtypes = [i64, P, i64, i32, i32, i32, P, i64, i32, P, P, i32]
            L.oracle_balance.argtypes = [i64, P, i64, i32, P, P]
            L.oracle_balance.restype = None
            L.oracle_precond_scaled.argtypes = [i64, P, i64, P, P, i32, P, P]
            L.oracle_precond_scaled.restype = None
            L.oracle_factor_scheme.restype = i32
            L.oracle_matvec_f32.argtypes = [i64, P, i64, P, P]
            L.oracle_matvec_f32.restype = None
            L.oracle_precond.argtypes = [i64, P, i64, P, P, i32]; L.oracle_precond.restype = None
            L.oracle_residual_vec.argtypes = [i64, P, i64, P, P, P]
            L.oracle_residual_vec.restype = None
            L.oracle_scaled_residual.argtypes = [i64, P, i64, P, i64, P, i64, i64, P]
            L.oracle_scaled_residual.restype = None
            L.oracle_solve_ir.argtypes = [i64, P, i64, P, i64, P, i64, P, i64, i64, i32, i32, d, d,
                                          d, i32, i32, P, P, ctypes.POINTER(IRInfo)]
            L.oracle_solve_ir.restype = i32
            L.oracle_num_threads.argtypes = []; L.oracle_num_threads.restype = i32
            L.oracle_set_num_threads.argtypes = [i32]; L.oracle_set_num_threads.restype = i32
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def round_to(x, fmt: int) -> np.ndarray:
    """Round fp64 values to a format (RNE), returned widened to fp64."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    y = np.empty_like(x)
    lib().oracle_round_array(_p(x), _p(y), x.size, fmt)
    return y


def lcg_jump(k: int) -> tuple[int, int]:
    a = ctypes.c_uint64(); c = ctypes.c_uint64()
    lib().oracle_lcg_jump(k, ctypes.byref(a), ctypes.byref(c))
    return a.value, c.value


def lcg_state(seed: int, t: int) -> int:
    return lib().oracle_lcg_state(seed, t)


def lcg_sequence(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    lib().oracle_lcg_sequence(seed, count, _p(out))
    return out


def draw_value(seed: int, t: int) -> float:
    return lib().oracle_draw_value(seed, t)


def generate(n: int, seed: int, margin: float = 1.0, mode: int = DOMINANT, nrhs: int = 1):
    """A (n x n, Fortran order) and b (n x nrhs) of the benchmark's system."""
    A = np.empty((n, n), dtype=np.float64, order="F")
    b = np.empty((n, max(nrhs, 0)), dtype=np.float64, order="F")
    rc = lib().oracle_generate(n, seed, margin, mode, _p(A), n, _p(b), n, nrhs)
    if rc != 0:
        raise ValueError("oracle_generate: bad arguments")
    return A, b


def generate_rows(n: int, seed: int, rows, margin: float = 1.0, mode: int = DOMINANT) -> np.ndarray:
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.empty((rows.size, n), dtype=np.float64)
    rc = lib().oracle_generate_rows(n, seed, margin, mode, _p(rows), rows.size, _p(out))
    if rc != 0:
        raise ValueError("oracle_generate_rows: bad arguments")
    return out


def _scales(rs, cs):
    if (rs is None) != (cs is None):
        raise ValueError("give both balancing scales or neither")
    if rs is None:
        return None, None, None
    rs = np.ascontiguousarray(np.asarray(rs, dtype=np.float64))
    cs = np.ascontiguousarray(np.asarray(cs, dtype=np.float64))
    return rs, cs, (_p(rs), _p(cs))


def balance(A, fmt: int = BF16) -> tuple[np.ndarray, np.ndarray]:
    """Power-of-two row / column balancing scales (rs, cs) of A for the format."""
    A = _f64(A)
    n = A.shape[0]
    rs = np.empty(n, dtype=np.float64)
    cs = np.empty(n, dtype=np.float64)
    lib().oracle_balance(n, _p(A), n, fmt, _p(rs), _p(cs))
    return rs, cs


def factor(A, fmt: int = BF16, nb: int = 128, fmt_update: int | None = None, rs=None,
           cs=None, trail32: bool = False) -> tuple[np.ndarray, int]:
    """Packed LU factors (widened to fp64) and 0 / 1 (zero or non-finite pivot);
    with balancing scales, of diag(rs) A diag(cs); trail32: Fig. 1 with a
    32-bit trailing matrix (fp32 Schur results, panels rounded to fmt once)."""
    A = _f64(A)
    n = A.shape[0]
    LU = np.empty((n, n), dtype=np.float64, order="F")
    rs, cs, ptrs = _scales(rs, cs)
    rc = lib().oracle_factor_scheme(n, _p(A), n, fmt, fmt if fmt_update is None else fmt_update, nb,
                                    _p(LU), n, 0, *(ptrs or (None, None)), int(trail32))
    if rc < 0:
        raise ValueError("oracle_factor: bad arguments")
    return LU, rc


def factor_plain(A, fmt: int = BF16, nb: int = 128) -> tuple[np.ndarray, int]:
    """The plain reading of Fig. 1: unblocked fp32 diagonal block of width nb,
    fp32 forward / back substitution for the panels, no inverses.  With
    fmt = FP64 the arithmetic is fp64 (nb 64 allowed: the fp64 study's LU)."""
    A = _f64(A)
    n = A.shape[0]
    LU = np.empty((n, n), dtype=np.float64, order="F")
    rc = lib().oracle_factor_scheme(n, _p(A), n, fmt, fmt, nb, _p(LU), n, 1, None, None, 0)
    if rc < 0:
        raise ValueError("oracle_factor_scheme: bad arguments")
    return LU, rc


def matvec_f32(A, v) -> np.ndarray:
    """The inner GMRES's fp32 Arnoldi product A v (A truncated toward zero to fp32)."""
    A = _f64(A)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    w = np.empty_like(v)
    lib().oracle_matvec_f32(A.shape[0], _p(A), A.shape[0], _p(v), _p(w))
    return w


def precond(LU, v, prec: int = 0, rs=None, cs=None) -> np.ndarray:
    LU = _f64(LU)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    z = np.empty_like(v)
    rs, cs, ptrs = _scales(rs, cs)
    lib().oracle_precond_scaled(LU.shape[0], _p(LU), LU.shape[0], _p(v), _p(z), prec, *(ptrs or (None, None)))
    return z


def residual_vec(A, x, b) -> np.ndarray:
    A = _f64(A)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    r = np.empty_like(b)
    lib().oracle_residual_vec(A.shape[0], _p(A), A.shape[0], _p(x), _p(b), _p(r))
    return r


def scaled_residual(A, X, B) -> np.ndarray:
    A = _f64(A)
    X = _f64(np.asarray(X).reshape(A.shape[0], -1))
    B = _f64(np.asarray(B).reshape(A.shape[0], -1))
    n, k = X.shape
    out = np.empty(k, dtype=np.float64)
    lib().oracle_scaled_residual(n, _p(A), n, _p(X), n, _p(B), n, k, _p(out))
    return out


def solve_ir(A, LU, B, restart: int = 30, max_iters: int = 50, inner_tol: float = 1e-12,
             theta: float = 0.1, accept: float = 16.0, precond_prec: int = 0, matvec_prec: int = 0,
             rs=None, cs=None):
    """GMRES-IR.  Returns (X, [info dict per rhs], worst status).
    precond_prec / matvec_prec: 1 = the inner GMRES's preconditioner / Arnoldi
    product in fp32, 0 = fp64.  rs, cs: the balancing scales the factors LU
    were computed with (both or neither)."""
    A = _f64(A)
    LU = _f64(LU)
    n = A.shape[0]
    B = _f64(np.asarray(B).reshape(n, -1))
    k = B.shape[1]
    X = np.zeros((n, k), dtype=np.float64, order="F")
    info = (IRInfo * k)()
    rc = lib().oracle_solve_ir(n, _p(A), n, _p(LU), n, _p(B), n, _p(X), n, k, restart, max_iters,
                               inner_tol, theta, accept, precond_prec, matvec_prec,
                               *(_scales(rs, cs)[2] or (None, None)), info)
    if rc < 0:
        raise ValueError("oracle_solve_ir: bad arguments")
    infos = [dict(iters=i.iters, outer=i.outer, scaled_resid=i.scaled_resid, status=i.status)
             for i in info]
    return X, infos, rc


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(k: int) -> int:
    """Threads of the oracle's parallel loops from now on; returns the number in effect."""
    return lib().oracle_set_num_threads(int(k))


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo), or the machine type."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        info = ""
    for key in ("model name", "Model Name", "Hardware"):
        for line in info.splitlines():
            if line.split(":")[0].strip() == key and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            parts.setdefault(k.strip(), v.strip())
    if "CPU implementer" in parts:
        return f"{platform.machine()} (implementer {parts['CPU implementer']}, part {parts.get('CPU part', '?')})"
    return platform.machine()


def split_lu(LU):
    """Unit-lower L and upper U from packed factors."""
    LU = np.asarray(LU)
    L = np.tril(LU, -1) + np.eye(LU.shape[0])
    U = np.triu(LU)
    return L, U
