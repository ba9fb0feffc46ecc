"""Serving workload: a stream of independent dense systems, each solved by the
HPL-MxP method (low-precision LU without pivoting + fp64 GMRES-IR), run by the
library's request executor (include/hpmxp_serve.h) with several requests in
flight on the GPU at once.

Requests: sizes n = floor(exp(U(ln 256, ln 8192))), 1..8 right-hand sides,
Poisson arrivals at `rate` per second, per-request generator seed
SplitMix64(stream_seed XOR id).  The matrices are the benchmark's own
generated systems (section "Matrix Generation"), made on the device inside
each request.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import capi
from .api import hpl_mxp_ops

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): one step from state x,
    i.e. the output for state x + golden gamma."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


@dataclass
class Spec:
    id: int
    n: int
    nrhs: int
    seed: int
    arrival: float   # seconds after the stream starts


def request_stream(count: int, rate: float, stream_seed: int = 2509, n_min: int = 256, n_max: int = 8192,
                   nrhs_max: int = 8) -> list[Spec]:
    rng = np.random.Generator(np.random.PCG64(stream_seed))
    gaps = rng.exponential(1.0 / rate, size=count) if rate > 0 else np.zeros(count)
    arrivals = np.cumsum(gaps) - (gaps[0] if count else 0.0)
    logn = rng.uniform(math.log(n_min), math.log(n_max), size=count)
    ns = np.clip(np.floor(np.exp(logn)).astype(np.int64), n_min, n_max)
    nrhs = rng.integers(1, nrhs_max + 1, size=count)
    return [Spec(i, int(ns[i]), int(nrhs[i]), splitmix64(stream_seed ^ i), float(arrivals[i])) for i in range(count)]


def make_request(spec: Spec, prec: int = capi.BF16, nb: int = 0, params: capi.IRParams | None = None,
                 x: torch.Tensor | None = None, margin: float = 1.0, diag: int = capi.DIAG_DOMINANT) -> capi.Request:
    """A request that generates its system on the device; x (a (nrhs, ldx)
    fp64 device tensor, column r = x[r]) receives the solution if given."""
    r = capi.Request()
    r.id, r.n, r.nrhs, r.prec, r.nb = spec.id, spec.n, spec.nrhs, prec, nb
    r.A, r.lda, r.b, r.ldb = None, 0, None, 0
    if x is not None:
        assert x.dtype == torch.float64 and x.shape[0] >= spec.nrhs and x.shape[1] >= spec.n
        r.x, r.ldx = x.data_ptr(), x.shape[1]
    else:
        r.x, r.ldx = None, 0
    r.seed, r.margin, r.diag_mode = spec.seed, margin, diag
    r.params = params if params is not None else capi.hpmxp_ir_params_default()
    return r


class Executor:
    """Owns the device arena (torch-allocated, once) and the native executor."""

    def __init__(self, workers: int = 8, arena_bytes: int = 16 << 30, device=None, batch: int = 1):
        """batch > 1: batch mode (hpmxp_executor_create_batched): each worker runs up
        to `batch` queued requests at once through the batched entry points."""
        dev = torch.device(device if device is not None else "cuda")
        index = dev.index if dev.index is not None else torch.cuda.current_device()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        torch.cuda.synchronize(dev)
        if batch > 1:
            st, h = capi.hpmxp_executor_create_batched(index, workers, batch, self.arena.data_ptr(),
                                                       int(arena_bytes))
        else:
            st, h = capi.hpmxp_executor_create(index, workers, self.arena.data_ptr(), int(arena_bytes))
        if st != capi.OK:
            raise capi.HpmxpError("hpmxp_executor_create", st)
        self.batch = batch
        self.h = h
        self.workers = workers
        self._buf = (capi.Completion * 256)()

    def submit(self, req: capi.Request):
        st = capi.hpmxp_executor_submit(self.h, req)
        if st != capi.OK:
            raise capi.HpmxpError("hpmxp_executor_submit", st)

    def poll(self, timeout_ms: int = 0) -> list[dict]:
        k = capi.hpmxp_executor_poll(self.h, self._buf, len(self._buf), int(timeout_ms))
        out = []
        for c in self._buf[:k]:
            out.append(dict(id=c.id, status=c.status, nrhs=c.nrhs, t_submit=c.t_submit, t_start=c.t_start,
                            t_done=c.t_done,
                            info=[dict(iters=c.info[r].iters, outer=c.info[r].outer,
                                       scaled_resid=c.info[r].scaled_resid, status=c.info[r].status)
                                  for r in range(c.nrhs)]))
        return out

    def outstanding(self) -> int:
        return capi.hpmxp_executor_outstanding(self.h)

    def close(self):
        if self.h:
            capi.hpmxp_executor_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_stream(ex: Executor, specs: list[Spec], prec: int = capi.BF16, params=None, xs=None, nb: int = 0,
               one_at_a_time: bool = False) -> list[dict]:
    """Submits every request at its arrival time (open loop) and collects the
    completions.  With one_at_a_time, each request is submitted only after the
    previous one completed (arrival times are then ignored)."""
    order = sorted(specs, key=lambda s: s.arrival)
    done: dict[int, dict] = {}
    t0 = time.perf_counter()
    i = 0
    while len(done) < len(order):
        if one_at_a_time:
            if i < len(order) and ex.outstanding() == 0:
                s = order[i]
                ex.submit(make_request(s, prec, nb, params, None if xs is None else xs[s.id]))
                i += 1
            for c in ex.poll(timeout_ms=100):
                done[c["id"]] = c
            continue
        now = time.perf_counter() - t0
        while i < len(order) and order[i].arrival <= now:
            s = order[i]
            ex.submit(make_request(s, prec, nb, params, None if xs is None else xs[s.id]))
            i += 1
        wait = 50 if i >= len(order) else int(max(0.0, order[i].arrival - now) * 1000)
        for c in ex.poll(timeout_ms=wait):
            done[c["id"]] = c
    return [done[s.id] for s in specs]


def summarize(specs: list[Spec], comps: list[dict], accept: float = 16.0) -> dict:
    lat = np.array([c["t_done"] - c["t_submit"] for c in comps])
    queue = np.array([c["t_start"] - c["t_submit"] for c in comps])
    t_first = min(c["t_submit"] for c in comps)
    t_last = max(c["t_done"] for c in comps)
    span = t_last - t_first
    ops = sum(hpl_mxp_ops(s.n, s.nrhs) for s in specs)
    ok = [c["status"] == capi.OK and all(i["scaled_resid"] < accept for i in c["info"]) for c in comps]
    valid = all(ok)
    statuses: dict[str, int] = {}
    for c in comps:
        name = capi.STATUS_NAMES.get(c["status"], str(c["status"]))
        statuses[name] = statuses.get(name, 0) + 1
    by_id = {s.id: s for s in specs}
    failed = [dict(id=c["id"], n=by_id[c["id"]].n, nrhs=by_id[c["id"]].nrhs, status=c["status"],
                   scaled_resid=[i["scaled_resid"] for i in c["info"]], iters=[i["iters"] for i in c["info"]])
              for c, good in zip(comps, ok) if not good]
    return dict(requests=len(comps), failed=len(failed), statuses=statuses, failed_examples=failed[:5],
                seconds=span, systems_per_s=len(comps) / span,
                tflops=ops / span / 1e12, p50_ms=float(np.percentile(lat, 50) * 1e3),
                p99_ms=float(np.percentile(lat, 99) * 1e3), mean_queue_ms=float(queue.mean() * 1e3),
                mean_iters=float(np.mean([i["iters"] for c in comps for i in c["info"]])),
                max_scaled_resid=float(max(i["scaled_resid"] for c in comps for i in c["info"])), valid=valid)
