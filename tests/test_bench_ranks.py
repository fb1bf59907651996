"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), each a
replica with its own problems; the job time is the slowest rank's and the
rate counts every rank's units.  No GPU: only the host-side aggregation runs."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    bench.barrier(w)
    t = bench.max_over_ranks(0.5 + rank, w)          # ranks took 0.5 s and 1.5 s
    q.put((r, lr, w, t, bench.job_rate(10, w, t)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 0, 2), (1, 1, 2)]
    for g in got:
        assert g[3] == 1.5                     # the slowest rank's time
        assert g[4] == pytest.approx(20 / 1.5)  # 10 units on each of 2 ranks


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.0, 1) == 2.0
    assert bench.job_rate(5, 1, 2.0) == 2.5
    bench.barrier(1)
