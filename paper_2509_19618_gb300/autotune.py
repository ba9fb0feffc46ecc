"""Autotuner for the factorization's schedule: the Schur-update depth nb in
{128, 256, 512} together with the library's schedule knobs (hpmxp_set_tuning):
the tile height of the 16-bit products (128 or 256 rows) and, where the
look-ahead schedule runs (n - 2 nb at least the overlap threshold), the SMs
reserved for the next panel chain (SMs / 16, / 10, / 6).

Each candidate is timed on the caller's matrix: one warm run, then the faster
of two timed runs.  The winner is applied (hpmxp_set_tuning) and cached per
(GPU name, n bucket, precision) in a JSON file under _build/, so later runs
skip the search.
"""
from __future__ import annotations

import itertools
import json
import os
from dataclasses import asdict, dataclass

import torch

from . import _build, api, capi

NB_CANDIDATES = (128, 256, 512)
TILE_CANDIDATES = (256, 128)
RESERVE_DIVISORS = (16, 10, 6)
OVERLAP_MIN_DEFAULT = 8192   # the library's built-in look-ahead threshold
CACHE = os.path.join(_build.BUILD, "autotune.json")
CACHE_VERSION = 2


@dataclass(frozen=True)
class Choice:
    nb: int
    gemm_tile: int = 0
    reserve_sms: int = 0

    def apply(self) -> None:
        """Set the tile height and reserve; the other knobs keep their values."""
        t = capi.hpmxp_get_tuning()
        t.update(gemm_tile=self.gemm_tile, reserve_sms=self.reserve_sms)
        api._check("hpmxp_set_tuning", capi.hpmxp_set_tuning(**t))


def _key(n: int, prec: int, device) -> str:
    bucket = 1 << max(8, (n - 1).bit_length())
    return f"v{CACHE_VERSION}|{torch.cuda.get_device_name(device)}|{bucket}|{prec}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def candidates(n: int, prec: int, sms: int) -> list[Choice]:
    """The search space for an order-n factorization on a GPU with `sms` SMs."""
    out = []
    for nb in NB_CANDIDATES:
        if nb > max(128, n):
            continue
        lookahead = prec not in (capi.BF16_TRAIL32, capi.FP16_TRAIL32) and n - 2 * nb >= OVERLAP_MIN_DEFAULT
        reserves = sorted({max(4, sms // d) for d in RESERVE_DIVISORS}) if lookahead else [0]
        # FP8 updates stay on the 128-row tile whatever the setting
        tiles = TILE_CANDIDATES if prec != capi.FP8_E4M3 else (0,)
        out += [Choice(nb, t, r) for t, r in itertools.product(tiles, reserves)]
    return out


def _time(choice: Choice, n: int, prec: int, A: api.ColMajor, device) -> float:
    choice.apply()
    LU = api.ColMajor.empty(n, n, api.factor_storage_dtype(prec), device)
    ws = api.workspace(capi.hpmxp_factor_workspace(n, prec, choice.nb), device)
    api.factor(A, prec, choice.nb, LU=LU, ws=ws)
    torch.cuda.synchronize(device)
    best = float("inf")
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.factor(A, prec, choice.nb, LU=LU, ws=ws)
        e1.record()
        torch.cuda.synchronize(device)
        best = min(best, e0.elapsed_time(e1))
    del LU, ws
    return best


def tune(n: int, prec: int, A: api.ColMajor, device="cuda", use_cache: bool = True) -> Choice:
    """Search (or recall) the fastest schedule for factoring A, apply it and return it."""
    key = _key(n, prec, device)
    cache = _load()
    if use_cache and key in cache:
        choice = Choice(**cache[key]["choice"])
        choice.apply()
        return choice
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    times = {}
    for c in candidates(n, prec, sms):
        times[c] = _time(c, n, prec, A, device)
    best = min(times, key=times.get)
    best.apply()
    cache[key] = {"choice": asdict(best),
                  "ms": [{**asdict(c), "ms": round(t, 4)} for c, t in sorted(times.items(), key=lambda kv: kv[1])]}
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best


def pick_nb(n: int, prec: int, A: api.ColMajor, device="cuda", use_cache: bool = True) -> int:
    """tune() for callers that only pass nb on: the schedule knobs are applied."""
    return tune(n, prec, A, device, use_cache).nb
