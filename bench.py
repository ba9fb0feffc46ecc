#!/usr/bin/env python
"""HPL-MxP benchmark on GB300: BF16 (or FP16 / FP8-update) LU without pivoting
+ fp64 GMRES-IR on the generated diagonally dominant system, reported as
HPL-MxP TFLOP/s = (2/3 n^3 + 3/2 n^2) / time-to-solution (section "Algorithmic
Framework").

One step = one full solve of the resident system: cast A to the factor format,
factor, x0 and GMRES-IR to scaled residual < 16.  Generation is untimed, as the
paper prescribes; the backward-error check runs after the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n 32768] [--nb 0|128|256|512] [--prec bf16|fp16|fp8]

Multi-GPU (torchrun, one rank per GPU): independent replicas of the same
solve, no collective on the data path; value = all ranks' work / max time.
`--impl reference` times the CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HPL-MxP TFLOP/s (2n^3/3 + 3n^2/2 per solve) at scaled residual < 16"
PREC = {"bf16": 0, "fp16": 1, "fp8": 2, "bf16t32": 3, "fp16t32": 4}


def hpl_ops(n: int) -> float:
    return 2.0 / 3.0 * n**3 + 1.5 * n**2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--nb", type=int, default=0, help="Schur update depth; 0 = autotune nb over 128/256/512 with the GEMM tile and reserved SMs")
    ap.add_argument("--prec", default="bf16", choices=list(PREC))
    ap.add_argument("--precond-fp32", type=int, default=1,
                    help="1: the preconditioner U^-1 L^-1 of the inner GMRES applied in fp32 (default), 0: fp64")
    ap.add_argument("--matvec-fp32", type=int, default=0,
                    help="1: the Arnoldi product A v of the inner GMRES in fp32, 0: fp64 (default)")
    ap.add_argument("--inner-tol", type=float, default=-1.0,
                    help="inner GMRES tolerance floor; -1: 1e-5 with an fp32 preconditioner, library default otherwise")
    ap.add_argument("--theta", type=float, default=-1.0,
                    help="adaptive inner-stopping factor of GMRES-IR; -1: the library default")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--diag", default="dominant", choices=["dominant", "sqrtn", "none"],
                    help="diagonal of the generated matrix (row sum + margin, sqrt(n) scaling, unscaled)")
    ap.add_argument("--margin", type=float, default=1.0, help="diagonal-dominance margin")
    ap.add_argument("--no-fp64-comparator", action="store_true",
                    help="skip the fp64 LU solve with partial pivoting (torch/cuSOLVER) of the same A")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variants: all-fp64 and all-fp32 inner operator, balanced (timed over --steps each)")
    ap.add_argument("--balance", type=int, default=0,
                    help="1: balance and scale A (hpmxp_balance) inside every timed solve")
    ap.add_argument("--serving-requests", type=int, default=600,
                    help="requests of the serving sub-record at 1000/s (a third of them at 100/s); 0: skip")
    ap.add_argument("--serving-batch", type=int, default=192, help="serving: requests per batch in batch mode")
    ap.add_argument("--serving-batch-workers", type=int, default=2, help="serving: workers in batch mode")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU oracle sample")
    ap.add_argument("--cpu-ladder", default="",
                    help="comma-separated n: time the CPU oracle alone at each (all cores, then one core up to "
                         "--cpu-ladder-single-max) and print one JSON line; no GPU work")
    ap.add_argument("--cpu-ladder-single-max", type=int, default=4096)
    ap.add_argument("--workload", default="solve", choices=["solve", "serving"],
                    help="solve: one large system (default); serving: a stream of small systems")
    ap.add_argument("--rate", type=float, default=1000.0, help="serving: Poisson arrival rate, requests/s")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests in the timed stream")
    ap.add_argument("--workers", type=int, default=12, help="serving: executor worker streams")
    ap.add_argument("--arena-gb", type=float, default=64.0, help="serving: executor arena (admission budget)")
    ap.add_argument("--serial-requests", type=int, default=300,
                    help="serving: requests of the one-at-a-time comparison (0: skip)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_setup(backend: str):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, local, ws


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(v: float, ws: int, device) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
IR_KW = {}   # refinement parameters of the GPU arm, mirrored by the oracle legs


def oracle_solve_timed(n: int, seed: int, prec: str, nb: int):
    import oracle
    A, b = oracle.generate(n, seed)
    fmt = oracle.FP16 if prec in ("fp16", "fp16t32") else oracle.BF16
    upd = oracle.E4M3 if prec == "fp8" else None
    t0 = time.perf_counter()
    LU, _ = oracle.factor(A, fmt, nb, fmt_update=upd, trail32=prec.endswith("t32"))
    X, info, rc = oracle.solve_ir(A, LU, b, **IR_KW)
    dt = time.perf_counter() - t0
    return dt, info[0], rc


def oracle_sample_size(target_s: float, seed: int, prec: str, nb: int) -> tuple[int, float]:
    """Largest multiple of 128 whose oracle solve should take about target_s."""
    n0 = 768
    dt, _, _ = oracle_solve_timed(n0, seed, prec, min(nb, 128))
    n = int(n0 * (target_s / max(dt, 1e-3)) ** (1 / 3)) // 128 * 128
    return max(256, min(n, 8192)), dt


def cpu_baseline(args, nb: int) -> dict:
    """The oracle on the host's cores (all of them, then one), each on a sample
    sized to about --cpu-seconds."""
    import oracle
    cores = oracle.num_threads()
    n, _ = oracle_sample_size(args.cpu_seconds, args.seed, args.prec, nb)
    dt, info, rc = oracle_solve_timed(n, args.seed, args.prec, min(nb, 512))
    single = None
    try:
        oracle.set_num_threads(1)
        n1, _ = oracle_sample_size(args.cpu_seconds / 2, args.seed, args.prec, nb)
        dt1, info1, rc1 = oracle_solve_timed(n1, args.seed, args.prec, min(nb, 512))
        single = {"value": hpl_ops(n1) / dt1 / 1e12, "unit": "TFLOP/s", "cores": 1,
                  "sample": f"one oracle solve at n={n1}, {dt1:.2f} s, status {rc1}, iters {info1['iters']}"}
    finally:
        oracle.set_num_threads(cores)
    return {"value": hpl_ops(n) / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "cpu_model": oracle.cpu_model(),
            "sample": f"one oracle solve (factor + GMRES-IR) of the same generated system at n={n} "
                      f"(the full n is out of reach on the host), {dt:.2f} s, status {rc}, iters {info['iters']}",
            "single_thread": single}


def run_cpu_ladder(args):
    """The oracle's own rate at several sizes on the host's cores: the ladder the
    one-sample cpu_baseline stands for, timed once per size (factor + GMRES-IR)."""
    import oracle
    cores = oracle.num_threads()
    nb = args.nb or 128
    rows = []
    for n in [int(v) for v in args.cpu_ladder.split(",") if v]:
        for threads in ([cores, 1] if n <= args.cpu_ladder_single_max else [cores]):
            oracle.set_num_threads(threads)
            dt, info, rc = oracle_solve_timed(n, args.seed, args.prec, min(nb, 512))
            rows.append({"n": n, "threads": threads, "seconds": dt, "tflops": hpl_ops(n) / dt / 1e12,
                         "status": rc, "iters": info["iters"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    oracle.set_num_threads(cores)
    print(json.dumps({"kind": "oracle ladder", "cpu_model": oracle.cpu_model(), "cores": cores, "nb": nb,
                      "prec": args.prec, "rows": rows}), flush=True)


SERVING_METRIC = "served systems/s (n log-uniform in [256, 8192], 1-8 rhs, Poisson arrivals), scaled residual < 16"


def serving_config(args, workers):
    return {"workload": f"serving: {args.requests} requests, n log-uniform 256..8192, nrhs 1..8, "
                        f"Poisson {args.rate:g}/s, stream seed 2509, {args.prec}",
            "rate": args.rate, "requests": args.requests, "workers": workers, "prec": args.prec,
            "parallelism": "replicas", "l2": "every request's A is new (generated on the device per request)"}


def run_reference_serving(args):
    import oracle
    from paper_2509_19618_gb300 import serve
    specs = serve.request_stream(args.requests, args.rate, stream_seed=2509)
    fmt = oracle.FP16 if args.prec == "fp16" else oracle.BF16
    upd = oracle.E4M3 if args.prec == "fp8" else None
    budget = max(5.0, min(60.0, 10.0 * max(1, args.steps)))
    done, ops, t = 0, 0.0, 0.0
    for s in specs:
        A, b = oracle.generate(s.n, s.seed, nrhs=s.nrhs)
        t0 = time.perf_counter()
        LU, _ = oracle.factor(A, fmt, 128 if s.n < 4096 else 256, fmt_update=upd)
        oracle.solve_ir(A, LU, b, **IR_KW)
        t += time.perf_counter() - t0
        done += 1
        ops += 2.0 / 3.0 * s.n**3 - 0.5 * s.n**2 + 2.0 * s.nrhs * s.n**2
        if t > budget:
            break
    value = done / t
    sample = f"the first {done} requests of the same stream, solved one at a time by the oracle ({t:.1f} s)"
    line = {"metric": SERVING_METRIC, "value": value, "unit": "systems/s", "n_gpus": args.gpus, "steps": done,
            "warmup": 0, "ms_per_step": t / done * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic (generated on the host by the oracle)",
            "impl": "reference", "config": serving_config(args, 1),
            "cpu_baseline": {"value": value, "unit": "systems/s", "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": sample, "tflops": ops / t / 1e12},
            "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args):
    rank, local, ws = dist_setup("nccl")
    import torch
    from paper_2509_19618_gb300 import capi, serve

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = PREC[args.prec]
    params = ir_params_for(args, args.precond_fp32, args.matvec_fp32)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    specs = serve.request_stream(args.requests, args.rate, stream_seed=2509 + rank)
    warm = serve.request_stream(max(3 * args.workers, 24), 0.0, stream_seed=1)
    with serve.Executor(workers=args.workers, arena_bytes=int(args.arena_gb * (1 << 30)), device=dev) as ex:
        serve.run_stream(ex, warm, prec, params)
        barrier(ws)
        launches0 = capi.hpmxp_launch_count()
        with ClockSampler(local) as clk:
            comps = serve.run_stream(ex, specs, prec, params)
        launches = capi.hpmxp_launch_count() - launches0
    summ = serve.summarize(specs, comps)
    span = allmax(summ["seconds"], ws, dev)
    serial = None
    if args.serial_requests > 0 and rank == 0:
        sub = specs[: args.serial_requests]
        with serve.Executor(workers=1, arena_bytes=int(args.arena_gb * (1 << 30)), device=dev) as ex1:
            c1 = serve.run_stream(ex1, sub, prec, params, one_at_a_time=True)
        s1 = serve.summarize(sub, c1)
        mixed_sub = serve.summarize(sub, [c for c in comps if c["id"] < len(sub)])
        serial = {"requests": len(sub), "systems_per_s": s1["systems_per_s"], "tflops": s1["tflops"],
                  "service_p50_ms": s1["p50_ms"], "service_p99_ms": s1["p99_ms"], "valid": s1["valid"],
                  "what": "the first requests of the stream, each submitted after the previous one completed "
                          "(one worker); latency here is service time only",
                  "mixed_p50_ms_same_requests": mixed_sub["p50_ms"]}
    if rank == 0:
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        tf = ws * summ["tflops"] * summ["seconds"] / span
        line = {"metric": SERVING_METRIC, "value": ws * args.requests / span, "unit": "systems/s", "n_gpus": ws,
                "steps": args.requests, "warmup": len(warm), "ms_per_step": span / args.requests * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
                "data": "synthetic (each request's system generated on the device from its seed)",
                "config": serving_config(args, args.workers),
                "valid": summ["valid"], "failed": summ["failed"], "statuses": summ["statuses"],
                "failed_examples": summ["failed_examples"], "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"],
                "mean_queue_ms": summ["mean_queue_ms"], "tflops": tf, "mean_ir_iters": summ["mean_iters"],
                "max_scaled_residual": summ["max_scaled_resid"], "one_at_a_time": serial,
                "gpu_launches": int(launches),
                "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                             "traffic": None, "kernel": "whole request mix (HPL-MxP operation count / wall time)"},
                "clocks": clk.summary(), "e2e": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    rank, local, ws = dist_setup("gloo")
    if rank != 0:
        return
    if args.workload == "serving":
        run_reference_serving(args)
        return
    import oracle
    nb = args.nb or 128
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    n, _ = oracle_sample_size(per_step, args.seed, args.prec, nb)
    for _ in range(args.warmup):
        oracle_solve_timed(n, args.seed, args.prec, nb)
    times = []
    for _ in range(args.steps):
        dt, info, rc = oracle_solve_timed(n, args.seed, args.prec, nb)
        times.append(dt)
    t = sum(times) / len(times)
    value = hpl_ops(n) / t / 1e12
    sample = f"oracle solve of the generated system at n={n} (nb={nb}, {args.prec}) per step"
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic (generated on the host by the oracle)",
            "impl": "reference",
            "config": {"workload": f"HPL-MxP solve, n={args.n} requested, sampled at n={n}", "n": n, "nb": nb,
                       "prec": args.prec, "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
GEMM_SRC = os.path.join(ROOT, "paper_2509_19618_gb300", "csrc", "gemm_tc.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gemm_tc_kernel_traffic_n32768_bf16_nb512.md")


def measured_gemm_traffic(n: int, nb: int, prec: str, gemm_tile: int):
    """DRAM bytes per gemm_tc_kernel launch over one solve, from the committed
    ncu summary of that workload (the library's default 256-row tile), or None
    when there is none for this workload and schedule or the kernel's source
    has changed since it was captured."""
    import hashlib
    if (n, nb, prec) != (32768, 512, "bf16") or gemm_tile not in (0, 256) or not os.path.exists(TRAFFIC_FILE):
        return None
    fields = {}
    for line in open(TRAFFIC_FILE):
        if line.startswith("traffic_") and ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    sha = hashlib.sha256(open(GEMM_SRC, "rb").read()).hexdigest()[:16]
    if fields.get("traffic_kernel_source_sha256_16") != sha:
        return None
    try:
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def ir_params_for(args, precond_fp32: int, matvec_fp32: int):
    from paper_2509_19618_gb300 import capi
    p = capi.hpmxp_ir_params_default()
    p.precond_fp32 = precond_fp32
    p.matvec_fp32 = matvec_fp32
    if args.inner_tol >= 0:
        p.inner_tol = args.inner_tol
    elif precond_fp32:
        p.inner_tol = 1e-5
    if args.theta >= 0:
        p.theta = args.theta
    return p


def operator_label(p) -> str:
    return (f"fp64 GMRES-IR(30): fp64 residual, MGS, Givens, update; preconditioner apply in "
            f"{'fp32' if p.precond_fp32 else 'fp64'}, Arnoldi product A v in {'fp32' if p.matvec_fp32 else 'fp64'}")


def time_solves(solver, A, b, steps: int, stream, dev):
    """Device time of `steps` whole solves (factor + GMRES-IR) on `stream`."""
    import torch
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    e0.record(stream)
    for _ in range(steps):
        x, info, st = solver(A, b)
        res.append((st, info[0]))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / 1e3 / steps, res


def serving_record(args, dev, params) -> dict:
    """Short serving runs of the request mix (n log-uniform 256..8192, 1-8 rhs):
    Poisson arrivals at 1000/s and 100/s, and the same requests one at a time."""
    from paper_2509_19618_gb300 import serve
    out = {"what": "request executor: each request generates its system on the device, factors it (BF16) and "
                   "refines it (fp64 GMRES-IR); requests are admitted by device footprint into a "
                   f"{args.arena_gb:g} GB arena and run on {args.workers} worker streams",
           "runs": []}
    warm = serve.request_stream(max(3 * args.workers, 24), 0.0, stream_seed=1)
    with serve.Executor(workers=args.workers, arena_bytes=int(args.arena_gb * (1 << 30)), device=dev) as ex:
        serve.run_stream(ex, warm, PREC[args.prec], params)
        for rate, count in ((1000.0, args.serving_requests), (100.0, max(1, args.serving_requests // 3))):
            specs = serve.request_stream(count, rate, stream_seed=2509)
            comps = serve.run_stream(ex, specs, PREC[args.prec], params)
            sm = serve.summarize(specs, comps)
            out["runs"].append({"rate": rate, "requests": count, "systems_per_s": sm["systems_per_s"],
                                "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"], "mean_queue_ms": sm["mean_queue_ms"],
                                "tflops": sm["tflops"], "valid": sm["valid"], "failed": sm["failed"],
                                "mean_ir_iters": sm["mean_iters"], "max_scaled_residual": sm["max_scaled_resid"]})
    # batch mode: each worker runs up to `serving_batch` queued requests through the batched
    # entry points (grouped factorization kernels, lockstep refinement)
    out["batched"] = []
    with serve.Executor(workers=args.serving_batch_workers, arena_bytes=int(args.arena_gb * (1 << 30)), device=dev,
                        batch=args.serving_batch) as exb:
        serve.run_stream(exb, warm, PREC[args.prec], params)
        for rate, count in ((1000.0, args.serving_requests), (100.0, max(1, args.serving_requests // 3))):
            specs = serve.request_stream(count, rate, stream_seed=2509)
            comps = serve.run_stream(exb, specs, PREC[args.prec], params)
            sm = serve.summarize(specs, comps)
            out["batched"].append({"rate": rate, "requests": count, "systems_per_s": sm["systems_per_s"],
                                   "p50_ms": sm["p50_ms"], "p99_ms": sm["p99_ms"],
                                   "mean_queue_ms": sm["mean_queue_ms"], "tflops": sm["tflops"],
                                   "valid": sm["valid"], "failed": sm["failed"],
                                   "workers": args.serving_batch_workers, "max_batch": args.serving_batch})
    sub = serve.request_stream(max(1, args.serving_requests // 3), 0.0, stream_seed=2509)
    with serve.Executor(workers=1, arena_bytes=int(args.arena_gb * (1 << 30)), device=dev) as ex1:
        c1 = serve.run_stream(ex1, sub, PREC[args.prec], params, one_at_a_time=True)
    s1 = serve.summarize(sub, c1)
    out["one_at_a_time"] = {"requests": len(sub), "systems_per_s": s1["systems_per_s"], "p50_ms": s1["p50_ms"],
                            "p99_ms": s1["p99_ms"], "valid": s1["valid"],
                            "what": "the first requests of the same stream, each submitted after the previous one "
                                    "completed (one worker): service time only"}
    return out


def main():
    args = parse()
    IR_KW.update(precond_prec=args.precond_fp32, matvec_prec=args.matvec_fp32,
                 inner_tol=args.inner_tol if args.inner_tol >= 0 else (1e-5 if args.precond_fp32 else 1e-12))
    if args.theta >= 0:
        IR_KW.update(theta=args.theta)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.cpu_ladder:
        run_cpu_ladder(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    rank, local, ws = dist_setup("nccl")
    import torch
    from paper_2509_19618_gb300 import api, autotune, capi

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, prec = args.n, PREC[args.prec]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    diag = {"dominant": capi.DIAG_DOMINANT, "sqrtn": capi.DIAG_SQRTN, "none": capi.DIAG_NONE}[args.diag]
    A, b = api.generate(n, seed=args.seed, margin=args.margin, diag=diag, device=dev)   # untimed (not timed by the paper)
    # the end-to-end leg's host copies of A and b, pinned up front (as a caller holding its data
    # in host memory would; api.HostBuffer: huge pages, registered with CUDA)
    # and the device buffers they are copied into, allocated and written once here (the first
    # copies into a newly allocated device buffer have measured far slower than later ones)
    host_in = dev_in = host_bufs = None
    if not args.no_e2e:
        host_bufs = (api.HostBuffer(A.storage.shape), api.HostBuffer(b.storage.shape))
        host_in = (host_bufs[0].tensor, host_bufs[1].tensor)
        host_in[0].copy_(A.storage)
        host_in[1].copy_(b.storage)
        dev_in = (api.ColMajor(torch.empty_like(A.storage), n, n), api.ColMajor(torch.empty_like(b.storage), n, 1))
        for _ in range(2):
            dev_in[0].storage.copy_(host_in[0], non_blocking=True)
            dev_in[1].storage.copy_(host_in[1], non_blocking=True)
        torch.cuda.synchronize(dev)
    params = ir_params_for(args, args.precond_fp32, args.matvec_fp32)
    if args.nb:
        schedule = {"nb": args.nb, **capi.hpmxp_get_tuning(), "source": "--nb flag, library defaults"}
        nb = args.nb
    else:
        choice = autotune.tune(n, prec, A, device=dev)
        nb = choice.nb
        schedule = {"nb": nb, "gemm_tile": choice.gemm_tile, "reserve_sms": choice.reserve_sms,
                    "source": "autotune (nb x GEMM tile x reserved SMs)"}
    fp64 = None
    if not args.no_fp64_comparator and rank == 0:
        # same system, fp64 LU with partial pivoting + solve (cuSOLVER through torch), one run after one warm-up
        Af = A.view().clone()
        bf = b.view().clone()
        LUw, pw = torch.linalg.lu_factor(Af[:1024, :1024])
        del LUw, pw
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        LUf, piv = torch.linalg.lu_factor(Af)
        xf = torch.linalg.lu_solve(LUf, piv, bf)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        xs = api.ColMajor.from_tensor(xf, dev)
        srf = float(api.residual(A, xs, b)[0])
        fp64 = {"value": hpl_ops(n) / (ms / 1e3) / 1e12, "unit": "TFLOP/s", "ms": ms, "scaled_residual": srf,
                "what": "torch.linalg.lu_factor + lu_solve (cuSOLVER, fp64, partial pivoting) on the same A, one run"}
        del Af, bf, LUf, piv, xf, xs
        torch.cuda.empty_cache()
    solver = api.Solver(n, 1, prec, nb, device=dev, params=params, balance=bool(args.balance))
    if not args.no_variants:
        # room for the fp32 copy of A that the all-fp32 variant's Arnoldi products read
        solver.sws = api.workspace(capi.hpmxp_solve_workspace(n, 1, params.restart) + capi.hpmxp_solve_workspace_a32(n),
                                   dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(args.warmup, 0)):
        solver(A, b)
    torch.cuda.synchronize(dev)

    capi.hpmxp_prof_enable(False)
    # timed region 1: device time of K whole solves, inputs resident in HBM
    launches0 = capi.hpmxp_launch_count()
    with ClockSampler(local) as clk:
        barrier(ws)
        t_step, infos = time_solves(solver, A, b, args.steps, stream, dev)
        barrier(ws)
    launches = capi.hpmxp_launch_count() - launches0
    t_step = allmax(t_step, ws, dev)
    ok = all(st == capi.OK for st, _ in infos)
    sr = float(api.residual(A, solver.x, b)[0])                 # untimed backward-error check
    if not ok or not sr < 16.0:
        print(f"warning: solve did not meet the HPL criterion (status {infos[-1][0]}, scaled residual {sr})",
              file=sys.stderr)
    value = ws * hpl_ops(n) / t_step / 1e12

    # per-kernel attribution: one more instrumented pass (events on the launching stream)
    capi.hpmxp_prof_reset()
    capi.hpmxp_prof_enable(True)
    solver(A, b)
    torch.cuda.synchronize(dev)
    capi.hpmxp_prof_enable(False)
    kinds = {"gemm_update": capi.PROF_GEMM, "gemm_panel": capi.PROF_GEMM_STORE, "gemv": capi.PROF_GEMV,
             "gemv32": capi.PROF_GEMV32, "precond": capi.PROF_PRECOND, "getrf": capi.PROF_GETRF,
             "cast": capi.PROF_CAST, "panel_ops": capi.PROF_PANEL, "balance": capi.PROF_BALANCE}
    prof = {k: capi.hpmxp_prof_read(v) for k, v in kinds.items()}
    # the GEMM launches' own execution time (first CTA start to last CTA end, global timer)
    dev_gemm = {k: capi.hpmxp_prof_read_device(kinds[k]) for k in ("gemm_update", "gemm_panel")}
    # every launch of the tensor-core GEMM kernel (Schur updates and panel products)
    g = {f: prof["gemm_update"][f] + prof["gemm_panel"][f] for f in ("ms", "work", "launches", "bytes")}
    g_dev_ms = sum(v["ms"] for v in dev_gemm.values())
    bf16_peak = peaks.get("bf16_tflops_sustained") or 1700.0
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    # achieved: flops per launch / the launch's average duration, the duration being the kernel's own
    # execution span; the look-ahead's four streams make the event interval around a launch include
    # the time it waits for SMs, reported beside it
    achieved = (g["work"] / (g_dev_ms / 1e3) / 1e12) if g_dev_ms > 0 else None
    achieved_ev = (g["work"] / (g["ms"] / 1e3) / 1e12) if g["ms"] > 0 else None
    peak = bf16_peak * (2.0 if prec == 2 else 1.0)
    # whole-solve roofline: 2/3 n^3 at the tensor peak plus 10 n^2 bytes per refinement
    # iteration (8 n^2 of A, 2 n^2 of factors) and once more for x0, at the HBM peak
    iters = infos[-1][1]["iters"]
    t_roof = (2.0 / 3.0 * n**3) / (peak * 1e12) + 10.0 * n * n * (iters + 1) / (hbm_peak * 1e9)
    roofline = {"bound": "tensor", "kernel": "gemm_tc_kernel (tcgen05 panel + Schur-update products)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": ("of measured: MEASURED_PEAKS.json bf16_tflops_sustained" if peaks
                                else "of fallback 1.7 PF/s") + (" x2 nominal fp8/bf16 ratio" if prec == 2 else ""),
                "frac": (achieved / peak) if achieved else None,
                "duration": "each launch's execution span on the device (global timer, first CTA start to "
                            "last CTA end), summed over the solve's launches",
                "achieved_event_interval": achieved_ev,
                "frac_event_interval": (achieved_ev / peak) if achieved_ev else None,
                "traffic": measured_gemm_traffic(n, nb, args.prec, schedule["gemm_tile"]),
                "algorithmic_bytes_per_launch": g["bytes"] / max(g["launches"], 1),
                # the same figure per role: the Schur updates carry the flops, the panel products
                # (substitution chains of 128-row products) are latency-bound; launches on the
                # look-ahead streams overlap, so their event durations include waiting for SMs
                "by_role": {role: {"launches": prof[kind]["launches"], "event_ms_per_solve": prof[kind]["ms"],
                                   "device_ms_per_solve": dev_gemm[kind]["ms"],
                                   "tflop_per_solve": prof[kind]["work"] / 1e12,
                                   "achieved_tflops": (prof[kind]["work"] / (dev_gemm[kind]["ms"] / 1e3) / 1e12
                                                       if dev_gemm[kind]["ms"] else None),
                                   "achieved_tflops_event_interval": (
                                       prof[kind]["work"] / (prof[kind]["ms"] / 1e3) / 1e12
                                       if prof[kind]["ms"] else None)}
                            for role, kind in (("schur_updates", "gemm_update"), ("panel_products", "gemm_panel"))},
                "whole_solve": {"t_roof_ms": t_roof * 1e3, "t_meas_ms": t_step * 1e3, "frac": t_roof / t_step,
                                "what": "T_roof = 2/3 n^3 / tensor peak + 10 n^2 (iters + 1) bytes / HBM peak"},
                "per_kind_ms_per_solve": {k: v["ms"] for k, v in prof.items()},
                "per_kind_launches": {k: v["launches"] for k, v in prof.items()}}
    gv = prof["gemv"]
    if gv["launches"]:
        roofline["gemv_gbs"] = gv["work"] / (gv["ms"] / 1e3) / 1e9
    pc = prof["precond"]
    if pc["launches"]:
        roofline["precond_gbs"] = pc["work"] / (pc["ms"] / 1e3) / 1e9
        roofline["precond_ms_per_apply"] = pc["ms"] / pc["launches"]

    # the same solve with other inner-operator precisions, over the same number of steps
    variants = {}
    if not args.no_variants:
        keep, keep_bal = solver.params, solver.balance
        x_head = solver.x.view().clone()
        legs = [("fp64_inner_operator", (0, 0), keep_bal), ("fp32_inner_operator", (1, 1), keep_bal),
                ("balanced" if not keep_bal else "unbalanced", (keep.precond_fp32, keep.matvec_fp32), not keep_bal)]
        for name, (pp, mp), bal in legs:
            if (pp, mp) == (keep.precond_fp32, keep.matvec_fp32) and bal == keep_bal:
                continue
            solver.params = ir_params_for(args, pp, mp)
            solver.balance = bal
            solver(A, b)
            t_v, res = time_solves(solver, A, b, args.steps, stream, dev)
            sr_v = float(api.residual(A, solver.x, b)[0])
            variants[name] = {"value": hpl_ops(n) / t_v / 1e12, "unit": "TFLOP/s", "ms_per_step": t_v * 1e3,
                              "steps": args.steps, "scaled_residual": sr_v,
                              "valid": bool(all(st == capi.OK for st, _ in res) and sr_v < 16.0),
                              "ir_iters": res[-1][1]["iters"], "ir_outer": res[-1][1]["outer"],
                              "what": operator_label(solver.params) +
                                      f", inner tolerance {solver.params.inner_tol:g}" +
                                      (", balancing and scaling (hpmxp_balance) inside the timed step" if bal
                                       else ", no balancing")}
            if name in ("balanced", "unbalanced"):
                variants[name]["x_bitwise_equal_to_headline"] = bool(torch.equal(solver.x.view(), x_head))
        solver.params, solver.balance = keep, keep_bal

    # timed region 2: end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        A_h, b_h = host_in
        x_h = torch.empty((1, solver.x.ld), dtype=torch.float64, pin_memory=True)
        A2, b2 = dev_in
        steps = max(1, min(args.steps, 5))

        def e2e_step(ev):
            ev[0].record()
            A2.storage.copy_(A_h, non_blocking=True)
            b2.storage.copy_(b_h, non_blocking=True)
            ev[1].record()
            solver(A2, b2)
            ev[2].record()
            x_h.copy_(solver.x.storage, non_blocking=True)
            torch.cuda.synchronize(dev)

        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps + 1)]
        e2e_warm = 3
        for _ in range(e2e_warm):   # untimed warm-up steps of the host path
            e2e_step(evs[0])
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(steps):
            e2e_step(evs[k + 1])
        t_e2e = (time.perf_counter() - t0) / steps
        h2d_ms = sum(e[0].elapsed_time(e[1]) for e in evs[1:]) / steps
        solve_ms = sum(e[1].elapsed_time(e[2]) for e in evs[1:]) / steps
        barrier(ws)
        t_e2e = allmax(t_e2e, ws, dev)
        serial = {"value": ws * hpl_ops(n) / t_e2e / 1e12, "unit": "TFLOP/s", "ms_per_step": t_e2e * 1e3,
                  "h2d_ms_per_step": h2d_ms, "solve_ms_per_step": solve_ms,
                  "what": "each step copies its inputs, then solves, then reads x back, one stream"}

        # pipelined: step k + 1's inputs are copied on a second stream into a second device
        # buffer while step k solves (double-buffered inputs), as a caller streaming systems
        # from host memory would run them; every step's copies and result read stay inside
        # the timed region
        A3 = api.ColMajor(torch.empty_like(A2.storage), n, n)
        b3 = api.ColMajor(torch.empty_like(b2.storage), n, 1)
        bufs = [(A2, b2), (A3, b3)]
        cstream = torch.cuda.Stream(dev)
        main = torch.cuda.current_stream(dev)

        def e2e_pipelined(nsteps):
            copied = [torch.cuda.Event(), torch.cuda.Event()]
            freed = [None, None]          # main-stream event after the last solve that read buffer i
            cev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nsteps)]

            def issue_copy(k):
                Ak, bk = bufs[k % 2]
                if freed[k % 2] is not None:
                    cstream.wait_event(freed[k % 2])
                cev[k][0].record(cstream)
                with torch.cuda.stream(cstream):
                    Ak.storage.copy_(A_h, non_blocking=True)
                    bk.storage.copy_(b_h, non_blocking=True)
                cev[k][1].record(cstream)
                copied[k % 2].record(cstream)

            issue_copy(0)
            for k in range(nsteps):
                main.wait_event(copied[k % 2])
                if k + 1 < nsteps:
                    issue_copy(k + 1)     # before the solve: the solve waits on the host for its decisions
                Ak, bk = bufs[k % 2]
                solver(Ak, bk)
                x_h.copy_(solver.x.storage, non_blocking=True)
                done = torch.cuda.Event()
                done.record(main)
                freed[k % 2] = done
            torch.cuda.synchronize(dev)
            return sum(e[0].elapsed_time(e[1]) for e in cev) / nsteps

        e2e_pipelined(e2e_warm)           # untimed warm-up steps
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        copy_ms = e2e_pipelined(steps)
        t_pipe = (time.perf_counter() - t0) / steps
        barrier(ws)
        t_pipe = allmax(t_pipe, ws, dev)
        x_ok = bool(torch.equal(x_h.view(-1)[:n], solver.x.storage.view(-1)[:n].cpu()))
        e2e = {"value": ws * hpl_ops(n) / t_pipe / 1e12, "unit": "TFLOP/s", "ms_per_step": t_pipe * 1e3,
               "h2d_bytes_per_step": int(A_h.numel() * 8 + b_h.numel() * 8),
               "d2h_bytes_per_step": int(x_h.numel() * 8), "steps": steps, "warmup": e2e_warm,
               "h2d_ms_per_step": copy_ms, "x_read_back_equal": x_ok,
               "what": "pipelined: the copy of step k+1's A and b (second stream, second device buffer) "
                       "overlaps the solve of step k; x read back every step; wall clock over all steps",
               "serial": serial}
        del A3, b3, bufs
        e2e["host_buffer"] = ("pinned (cudaHostRegister) anonymous mapping, " +
                              ("transparent huge pages" if host_bufs[0].huge_pages else "base pages"))
        del A_h, b_h, x_h, A2, b2, host_in, dev_in
        for hb in host_bufs:
            hb.close()
    del A, b, solver
    torch.cuda.empty_cache()

    serving = None
    if args.serving_requests > 0 and rank == 0:
        serving = serving_record(args, dev, ir_params_for(args, args.precond_fp32, args.matvec_fp32))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, nb)

    if rank == 0:
        speedup = (value / fp64["value"]) if fp64 else None
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.prec, "data": "synthetic (on-device LCG generator, seed %d)"
                % args.seed,
                "config": {"workload": f"HPL-MxP single system n={n}, {args.prec} LU nb={nb} + "
                                       + operator_label(params),
                           "n": n, "nb": nb, "prec": args.prec, "global_batch": ws, "seq_len": None,
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (A is %.1f GB)" % (8 * n * n / 1e9),
                           "precond_fp32": int(params.precond_fp32), "matvec_fp32": int(params.matvec_fp32),
                           "inner_tol": params.inner_tol, "balance": int(args.balance), "schedule": schedule},
                "valid": bool(ok and sr < 16.0), "scaled_residual": sr,
                "ir_iters": infos[-1][1]["iters"], "ir_outer": infos[-1][1]["outer"],
                "ir_status": int(infos[-1][0]), "diag": args.diag, "margin": args.margin,
                "fp64_lu_comparator": fp64, "speedup_vs_fp64_lu": speedup, "variants": variants,
                "serving": serving, "gpu_launches": int(launches), "roofline": roofline, "clocks": clk.summary(),
                "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
