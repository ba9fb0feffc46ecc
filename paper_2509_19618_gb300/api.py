"""PyTorch-facing wrappers over the C interface: device memory and streams
come from torch, every step of the solve runs in libhpmxp.so.

Matrices are column major: a ``ColMajor`` keeps a (cols x ld) torch tensor
whose row j is column j of the matrix, so element (i, j) lives at
``storage[j, i]`` and ``ColMajor.view()`` is the (rows x cols) matrix.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import capi


def _round_up(a: int, b: int) -> int:
    return (a + b - 1) // b * b


def stream_handle(stream: torch.cuda.Stream | None = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class ColMajor:
    storage: torch.Tensor   # (cols, ld)
    rows: int
    cols: int

    @property
    def ld(self) -> int:
        return self.storage.shape[1]

    @property
    def ptr(self) -> int:
        return self.storage.data_ptr()

    def view(self) -> torch.Tensor:
        return self.storage[:, : self.rows].t()

    @staticmethod
    def empty(rows: int, cols: int, dtype, device, ld: int | None = None, align: int = 8) -> "ColMajor":
        ld = ld if ld is not None else _round_up(max(rows, 1), align)
        return ColMajor(torch.empty((cols, ld), dtype=dtype, device=device), rows, cols)

    @staticmethod
    def from_tensor(t: torch.Tensor, device, dtype=torch.float64, align: int = 8) -> "ColMajor":
        t = torch.as_tensor(t)
        if t.dim() == 1:
            t = t[:, None]
        m = ColMajor.empty(t.shape[0], t.shape[1], dtype, device, align=align)
        m.view().copy_(t.to(device=device, dtype=dtype))
        return m


class HostBuffer:
    """Page-locked host memory for a caller that keeps its inputs on the host.

    An anonymous mapping advised for transparent huge pages (512 MiB on an Arm
    kernel with 64 KiB base pages, 2 MiB on x86-64), filled once so its pages
    exist, then registered with CUDA.  With huge pages a multi-GB copy needs a
    few address translations instead of one per base page.  Where the kernel
    refuses the advice the buffer is still pinned, on base pages.
    ``tensor`` is a CPU tensor of the given shape over the mapping; ``close()``
    (or garbage collection) unregisters and unmaps it.
    """

    def __init__(self, shape, dtype=torch.float64):
        import mmap
        self.shape = tuple(int(d) for d in shape)
        numel = int(np.prod(self.shape)) if self.shape else 1
        if numel <= 0:
            raise ValueError(f"HostBuffer of shape {self.shape} holds no elements")
        self.nbytes = numel * torch.empty((), dtype=dtype).element_size()
        self._map = mmap.mmap(-1, self.nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        self.huge_pages = False
        if hasattr(mmap, "MADV_HUGEPAGE"):
            try:
                self._map.madvise(mmap.MADV_HUGEPAGE)
                self.huge_pages = True
            except OSError:
                pass
        flat = torch.frombuffer(self._map, dtype=dtype, count=numel)
        flat.zero_()
        self.tensor = flat.view(self.shape)
        err = torch.cuda.cudart().cudaHostRegister(flat.data_ptr(), self.nbytes, 0)
        if int(err) != 0:
            self.tensor = None
            self._map.close()
            raise RuntimeError(f"cudaHostRegister failed ({err}) for {self.nbytes} bytes")
        self._registered = True

    def close(self):
        if getattr(self, "_registered", False):
            torch.cuda.cudart().cudaHostUnregister(self.tensor.data_ptr())
            self._registered = False
        self.tensor = None
        if getattr(self, "_map", None) is not None:
            try:
                self._map.close()
            except BufferError:   # a view of the tensor is still alive: the mapping goes with it
                pass
            self._map = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _check(fn: str, status: int):
    if status != capi.OK:
        raise capi.HpmxpError(fn, status)


def generate(n: int, seed: int = 1, margin: float = 1.0, diag: int = capi.DIAG_DOMINANT, nrhs: int = 1,
             device="cuda", stream=None) -> tuple[ColMajor, ColMajor]:
    """The benchmark's system A (n x n fp64) and b (n x nrhs fp64), generated on the device."""
    A = ColMajor.empty(n, n, torch.float64, device)
    b = ColMajor.empty(n, max(nrhs, 1), torch.float64, device)
    ws = workspace(capi.hpmxp_generate_workspace(n), device)
    st = capi.hpmxp_generate(n, seed, margin, diag, A.ptr, A.ld, b.ptr, b.ld, nrhs, ws.data_ptr(), ws.numel(),
                             stream_handle(stream))
    _check("hpmxp_generate", st)
    return A, b


def factor_storage_dtype(prec: int):
    return torch.float16 if prec in (capi.FP16, capi.FP16_TRAIL32) else torch.bfloat16


def balance(A: ColMajor, prec: int = capi.BF16, scales: tuple | None = None, stream=None):
    """Power-of-two balancing scales (rs, cs) of A for the factor format, as two
    fp64 device tensors of n entries (hpmxp_balance)."""
    n = A.rows
    rs, cs = scales if scales is not None else (torch.empty(n, dtype=torch.float64, device=A.storage.device),
                                                torch.empty(n, dtype=torch.float64, device=A.storage.device))
    _check("hpmxp_balance", capi.hpmxp_balance(n, A.ptr, A.ld, prec, rs.data_ptr(), cs.data_ptr(),
                                               stream_handle(stream)))
    return rs, cs


def _scale_ptrs(scales):
    if scales is None:
        return None, None
    return scales[0].data_ptr(), scales[1].data_ptr()


def factor(A: ColMajor, prec: int = capi.BF16, nb: int = 128, LU: ColMajor | None = None, ws=None,
           stream=None, check: bool = True, scales: tuple | None = None) -> ColMajor:
    """Low-precision LU without pivoting of A (of diag(rs) A diag(cs) with
    scales = (rs, cs) from `balance`); returns the packed factors.
    With check=False a breakdown status is left in `factor.last_status` instead of raising."""
    n = A.rows
    if LU is None:
        LU = ColMajor.empty(n, n, factor_storage_dtype(prec), A.storage.device)
    if ws is None:
        ws = workspace(capi.hpmxp_factor_workspace(n, prec, nb), A.storage.device)
    rs, cs = _scale_ptrs(scales)
    st = capi.hpmxp_factor_scaled(n, A.ptr, A.ld, prec, nb, rs, cs, LU.ptr, LU.ld, ws.data_ptr(), ws.numel(),
                                  stream_handle(stream))
    factor.last_status = st
    if check or st not in (capi.OK, capi.EBREAKDOWN):
        _check("hpmxp_factor", st)
    return LU


def ir_params(**kw) -> capi.IRParams:
    p = capi.hpmxp_ir_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def solve_ir(A: ColMajor, LU: ColMajor, b: ColMajor, prec: int = capi.BF16, params: capi.IRParams | None = None,
             x: ColMajor | None = None, ws=None, stream=None, check: bool = True, scales: tuple | None = None):
    """GMRES-IR (with the factors of the balanced matrix when scales = (rs, cs));
    returns (x, [info dicts], status)."""
    n, k = A.rows, b.cols
    if x is None:
        x = ColMajor.empty(n, k, torch.float64, A.storage.device)
    restart = params.restart if params is not None else 30
    if ws is None:
        ws = workspace(capi.hpmxp_solve_workspace(n, k, restart), A.storage.device)
    info = (capi.IRInfo * k)()
    rs, cs = _scale_ptrs(scales)
    st = capi.hpmxp_solve_ir_scaled(n, A.ptr, A.ld, LU.ptr, LU.ld, prec, rs, cs, b.ptr, b.ld, x.ptr, x.ld, k,
                                    params, info, ws.data_ptr(), ws.numel(), stream_handle(stream))
    infos = [dict(iters=i.iters, outer=i.outer, scaled_resid=i.scaled_resid, status=i.status) for i in info]
    if check and st not in (capi.OK, capi.ENOCONV, capi.EBREAKDOWN):
        _check("hpmxp_solve_ir", st)
    return x, infos, st


def residual(A: ColMajor, x: ColMajor, b: ColMajor, stream=None) -> np.ndarray:
    """HPL scaled residual of every column (fp64, on the device)."""
    n, k = A.rows, x.cols
    out = (ctypes.c_double * k)()
    ws = workspace(capi.hpmxp_residual_workspace(n, k), A.storage.device)
    st = capi.hpmxp_residual(n, A.ptr, A.ld, x.ptr, x.ld, b.ptr, b.ld, k, ctypes.addressof(out), ws.data_ptr(),
                             ws.numel(), stream_handle(stream))
    _check("hpmxp_residual", st)
    return np.array(out[:], dtype=np.float64)


def _problem(A: ColMajor, LU: ColMajor, b: ColMajor | None = None, x: ColMajor | None = None) -> capi.Problem:
    p = capi.Problem()
    p.n, p.A, p.lda, p.LU, p.ldlu = A.rows, A.ptr, A.ld, LU.ptr, LU.ld
    if b is not None:
        p.b, p.ldb, p.x, p.ldx, p.nrhs = b.ptr, b.ld, x.ptr, x.ld, b.cols
    return p


def factor_batched(As: list, prec: int = capi.BF16, LUs: list | None = None, stream=None, check: bool = True):
    """Factors every system of the list in one batched call (depth 128, grouped
    kernels); returns (factors, per-system statuses)."""
    dev = As[0].storage.device
    if LUs is None:
        LUs = [ColMajor.empty(A.rows, A.rows, factor_storage_dtype(prec), dev) for A in As]
    probs = [_problem(A, LU) for A, LU in zip(As, LUs)]
    ws = workspace(capi.hpmxp_factor_batched_workspace(probs, prec), dev)
    st, per = capi.hpmxp_factor_batched(probs, prec, ws.data_ptr(), ws.numel(), stream_handle(stream))
    if check and st not in (capi.OK, capi.EBREAKDOWN):
        _check("hpmxp_factor_batched", st)
    return LUs, per


def solve_ir_batched(As: list, LUs: list, bs: list, prec: int = capi.BF16, params: capi.IRParams | None = None,
                     xs: list | None = None, stream=None, check: bool = True):
    """GMRES-IR of every system in lockstep; returns (solutions, [per-system info lists], status)."""
    dev = As[0].storage.device
    if xs is None:
        xs = [ColMajor.empty(A.rows, b.cols, torch.float64, dev) for A, b in zip(As, bs)]
    probs = [_problem(A, LU, b, x) for A, LU, b, x in zip(As, LUs, bs, xs)]
    restart = params.restart if params is not None else 30
    ws = workspace(capi.hpmxp_solve_ir_batched_workspace(probs, restart), dev)
    total = sum(b.cols for b in bs)
    info = (capi.IRInfo * total)()
    st = capi.hpmxp_solve_ir_batched(probs, prec, params, info, ws.data_ptr(), ws.numel(), stream_handle(stream))
    if check and st not in (capi.OK, capi.ENOCONV, capi.EBREAKDOWN):
        _check("hpmxp_solve_ir_batched", st)
    infos, off = [], 0
    for b in bs:
        infos.append([dict(iters=i.iters, outer=i.outer, scaled_resid=i.scaled_resid, status=i.status)
                      for i in info[off:off + b.cols]])
        off += b.cols
    return xs, infos, st


def hpl_mxp_ops(n: int, nrhs: int = 1) -> float:
    """Canonical operation count (section "Algorithmic Framework"): 2/3 n^3 + 3/2 n^2
    for one right-hand side; with k right-hand sides the solves count 2 k n^2."""
    return 2.0 / 3.0 * n**3 - 0.5 * n**2 + 2.0 * nrhs * n**2


class Solver:
    """Reusable device buffers for repeated solves of one shape (bench, serving)."""

    def __init__(self, n: int, nrhs: int = 1, prec: int = capi.BF16, nb: int = 128, device="cuda",
                 params: capi.IRParams | None = None, balance: bool = False):
        self.n, self.nrhs, self.prec, self.nb = n, nrhs, prec, nb
        self.balance = balance   # balancing and scaling as part of every solve (hpmxp_balance)
        self.params = params if params is not None else capi.hpmxp_ir_params_default()
        self.device = torch.device(device)
        self.LU = ColMajor.empty(n, n, factor_storage_dtype(prec), self.device)
        self.x = ColMajor.empty(n, nrhs, torch.float64, self.device)
        self.fws = workspace(capi.hpmxp_factor_workspace(n, prec, nb), self.device)
        # with fp32 Arnoldi products, room for their fp32 copy of A (half the bytes per product)
        extra = capi.hpmxp_solve_workspace_a32(n) if self.params.matvec_fp32 else 0
        self.sws = workspace(capi.hpmxp_solve_workspace(n, nrhs, self.params.restart) + extra, self.device)
        self.scales = (torch.empty(n, dtype=torch.float64, device=self.device),
                       torch.empty(n, dtype=torch.float64, device=self.device))

    def factor(self, A: ColMajor, stream=None) -> ColMajor:
        sc = balance(A, self.prec, self.scales, stream) if self.balance else None
        LU = factor(A, self.prec, self.nb, LU=self.LU, ws=self.fws, stream=stream, check=False, scales=sc)
        self.factor_status = factor.last_status
        return LU

    def solve(self, A: ColMajor, b: ColMajor, stream=None):
        return solve_ir(A, self.LU, b, self.prec, self.params, x=self.x, ws=self.sws, stream=stream,
                        scales=self.scales if self.balance else None)

    def __call__(self, A: ColMajor, b: ColMajor, stream=None):
        self.factor(A, stream)
        return self.solve(A, b, stream)
