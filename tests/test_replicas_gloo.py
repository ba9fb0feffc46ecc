"""The multi-GPU path of bench.py is replicas only: each rank solves its own
system, the ranks meet at a barrier around the timed region, and rank 0
reports all ranks' work over the slowest rank's time.  This checks that host
logic with two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, local, ws = bench.dist_setup("gloo")
    bench.barrier(ws)
    t = 1.0 + rank          # rank 1 is the slow one
    tmax = bench.allmax(t, ws, "cpu")
    n = 1000
    value = ws * bench.hpl_ops(n) / tmax
    bench.barrier(ws)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, ws, tmax, value))


def test_two_gloo_ranks_report_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    for r, ws, tmax, value in out:
        assert ws == 2 and tmax == 2.0
        assert value == pytest.approx(2 * bench.hpl_ops(1000) / 2.0)
    assert [o[0] for o in out] == [0, 1]
