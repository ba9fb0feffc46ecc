"""Autotuner for the Schur-update depth nb in {128, 256, 512}.

Times one factorization per candidate on the caller's matrix (after one warm
run each) and keeps the fastest; results are cached per (GPU name, n bucket,
precision) in a JSON file under _build/ so later runs skip the search.
"""
from __future__ import annotations

import json
import os

import torch

from . import _build, api

CANDIDATES = (128, 256, 512)
CACHE = os.path.join(_build.BUILD, "autotune.json")


def _key(n: int, prec: int, device) -> str:
    bucket = 1 << max(8, (n - 1).bit_length())
    return f"{torch.cuda.get_device_name(device)}|{bucket}|{prec}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def pick_nb(n: int, prec: int, A: api.ColMajor, device="cuda", use_cache: bool = True) -> int:
    key = _key(n, prec, device)
    cache = _load()
    if use_cache and key in cache:
        return int(cache[key]["nb"])
    times = {}
    for nb in CANDIDATES:
        if nb > max(128, n):
            continue
        LU = api.ColMajor.empty(n, n, api.factor_storage_dtype(prec), device)
        ws = api.workspace(api.capi.hpmxp_factor_workspace(n, prec, nb), device)
        api.factor(A, prec, nb, LU=LU, ws=ws)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.factor(A, prec, nb, LU=LU, ws=ws)
        e1.record()
        torch.cuda.synchronize(device)
        times[nb] = e0.elapsed_time(e1)
        del LU, ws
    best = min(times, key=times.get)
    cache[key] = {"nb": best, "ms": times}
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best
