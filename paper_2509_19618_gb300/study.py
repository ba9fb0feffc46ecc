"""Pivot growth and residual norms of 64-bit LU with and without partial
pivoting (section "Experimental Results", Figs. 2-4).

For each generated system this measures, on the GPU:
  * the library's fp64 LU WITHOUT pivoting (hpmxp_lu_f64) and its solve;
  * fp64 LU WITH partial pivoting (GEPP) and its solve, from cuSOLVER through
    torch.linalg.lu_factor / lu_solve, the library call the paper compares
    against;
and reports, for both, the largest pivot |u_kk| and where it occurs (as a
fraction of n), the growth max|U| / max|A|, and the 1-, 2- and inf-norms of the
residual r = b - A x together with the backward errors
||r|| / ((||A|| ||x|| + ||b||) n eps) in each norm (eps = 2^-53; for the
2-norm, ||A||_2 is bounded by sqrt(||A||_1 ||A||_inf)).  The residual is the
library's fp64 GEMV (hpmxp_residual_vector).

Matrices: the benchmark's generator; `unit_range` doubles every entry (exact)
so that the raw draws are uniform in (-1, 1) as in the paper's figures.
Reference curves of Fig. 2: sqrt(n), 5/8 sqrt(n) and n^0.45.

  python -m paper_2509_19618_gb300.study --sizes 1024,2048,4096 --seeds 3 --modes none,sqrtn
"""
from __future__ import annotations

import argparse
import json
import math
import time

import torch

from . import api, capi

EPS = 2.0**-53
MODES = {"dominant": capi.DIAG_DOMINANT, "sqrtn": capi.DIAG_SQRTN, "none": capi.DIAG_NONE,
         "departure": capi.DIAG_DEPARTURE}


def lu_f64(A: api.ColMajor, stream=None) -> tuple[api.ColMajor, int]:
    """fp64 LU without pivoting of a copy of A: (packed factors, status)."""
    LU = api.ColMajor(A.storage.clone(), A.rows, A.cols)
    ws = api.workspace(capi.hpmxp_lu_f64_workspace(A.rows), A.storage.device)
    st = capi.hpmxp_lu_f64(A.rows, LU.ptr, LU.ld, ws.data_ptr(), ws.numel(), api.stream_handle(stream))
    return LU, st


def lu_solve_f64(LU: api.ColMajor, b: api.ColMajor, stream=None) -> api.ColMajor:
    x = api.ColMajor(b.storage.clone(), b.rows, b.cols)
    st = capi.hpmxp_lu_solve_f64(LU.rows, LU.ptr, LU.ld, x.ptr, x.ld, b.cols, api.stream_handle(stream))
    api._check("hpmxp_lu_solve_f64", st)
    return x


def residual_vector(A: api.ColMajor, x: api.ColMajor, b: api.ColMajor, stream=None) -> api.ColMajor:
    n, k = A.rows, x.cols
    r = api.ColMajor.empty(n, k, torch.float64, A.storage.device)
    ws = api.workspace(capi.hpmxp_residual_workspace(n, k), A.storage.device)
    st = capi.hpmxp_residual_vector(n, A.ptr, A.ld, x.ptr, x.ld, b.ptr, b.ld, k, r.ptr, r.ld, ws.data_ptr(),
                                    ws.numel(), api.stream_handle(stream))
    api._check("hpmxp_residual_vector", st)
    return r


def _norms(Av: torch.Tensor, xv: torch.Tensor, bv: torch.Tensor, rv: torch.Tensor, a_norms: dict) -> dict:
    n = Av.shape[0]
    out = {}
    for name, p in (("1", 1), ("2", 2), ("inf", math.inf)):
        rn = float(torch.linalg.vector_norm(rv, p))
        xn = float(torch.linalg.vector_norm(xv, p))
        bn = float(torch.linalg.vector_norm(bv, p))
        out[f"r_{name}"] = rn
        out[f"backward_{name}"] = rn / ((a_norms[name] * xn + bn) * n * EPS)
    return out


def _pivots(U_diag: torch.Tensor, U_absmax: float, a_max: float) -> dict:
    piv = U_diag.abs()
    k = int(torch.argmax(piv))
    n = piv.numel()
    return {"max_pivot": float(piv[k]), "max_pivot_at": k, "max_pivot_pos": (k + 1) / n,
            "growth": U_absmax / a_max}


def run_case(n: int, seed: int, mode: str = "none", margin: float = 1.0, unit_range: bool = True,
             device="cuda") -> dict:
    dev = torch.device(device)
    A, b = api.generate(n, seed=seed, margin=margin, diag=MODES[mode], device=dev)
    if unit_range:
        A.view().mul_(2.0)
        b.view().mul_(2.0)
    Av, bv = A.view(), b.view()[:, 0]
    a_max = float(Av.abs().max())
    a1 = float(Av.abs().sum(dim=0).max())
    ainf = float(Av.abs().sum(dim=1).max())
    a_norms = {"1": a1, "inf": ainf, "2": math.sqrt(a1 * ainf)}
    rec = {"n": n, "seed": seed, "mode": mode, "margin": margin, "unit_range": unit_range,
           "ref_sqrt_n": math.sqrt(n), "ref_5_8_sqrt_n": 0.625 * math.sqrt(n), "ref_n_045": n**0.45}
    # without pivoting (this library's fp64 LU)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    LU, st = lu_f64(A)
    rec["nopiv_status"] = capi.STATUS_NAMES.get(st, st)
    x = lu_solve_f64(LU, b)
    torch.cuda.synchronize(dev)
    rec["nopiv_seconds"] = time.perf_counter() - t0
    r = residual_vector(A, x, b)
    U = torch.triu(LU.view())
    rec["nopiv"] = {**_pivots(torch.diagonal(LU.view()), float(U.abs().max()), a_max),
                    **_norms(Av, x.view()[:, 0], bv, r.view()[:, 0], a_norms)}
    del LU, U, x, r
    # with partial pivoting (cuSOLVER getrf / getrs through torch)
    t0 = time.perf_counter()
    LUp, piv = torch.linalg.lu_factor(Av)
    xp = torch.linalg.lu_solve(LUp, piv, b.view())
    torch.cuda.synchronize(dev)
    rec["gepp_seconds"] = time.perf_counter() - t0
    xs = api.ColMajor.from_tensor(xp, dev)
    r = residual_vector(A, xs, b)
    Up = torch.triu(LUp)
    rec["gepp"] = {**_pivots(torch.diagonal(LUp), float(Up.abs().max()), a_max),
                   **_norms(Av, xs.view()[:, 0], bv, r.view()[:, 0], a_norms)}
    del LUp, piv, xp, xs, Up, r, A, b
    torch.cuda.empty_cache()
    return rec


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--sizes", default="1024,2048,4096,8192")
    ap.add_argument("--seeds", type=int, default=3, help="seeds 1..S per size")
    ap.add_argument("--modes", default="none,sqrtn,departure", help=",".join(MODES))
    ap.add_argument("--margin", type=float, default=1.0, help="SQRTN coefficient / DEPARTURE ratio")
    ap.add_argument("--out", default="", help="also write the JSON lines here")
    args = ap.parse_args(argv)
    recs = []
    for mode in args.modes.split(","):
        margin = args.margin if mode != "departure" or args.margin != 1.0 else 0.9
        for n in [int(v) for v in args.sizes.split(",")]:
            for seed in range(1, args.seeds + 1):
                rec = run_case(n, seed, mode, margin)
                recs.append(rec)
                print(json.dumps(rec), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            for rec in recs:
                f.write(json.dumps(rec) + "\n")


if __name__ == "__main__":
    main()
