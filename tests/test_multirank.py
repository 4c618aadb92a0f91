"""The N > 1 path of bench.py on two CPU ranks (gloo, 127.0.0.1).

With several GPUs bench.py runs one independent replica of the workload per
rank (the path has no data exchange between problems), times each with
barriers on both sides, takes the slowest rank's time and reports the units
of all ranks per second of it.  The host logic is checked here without a GPU:
the barrier, the max over ranks and the whole-job rate.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench.barrier(ws)
    t = bench.max_over_ranks(ws, 1.0 + rank)  # rank 1 is the slow one
    rate = bench.whole_job_rate(1000, ws, 10, t)
    bench.barrier(ws)
    dist.destroy_process_group()
    out.put((rank, t, rate))


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, rate in res:
        assert t == pytest.approx(2.0)  # the max over ranks
        assert rate == pytest.approx(1000 * 2 * 10 / 2.0)  # all ranks' units per slowest second


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert bench.whole_job_rate(10, 1, 4, 2.0) == 20.0
