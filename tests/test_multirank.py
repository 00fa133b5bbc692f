"""The replicas-only multi-GPU path of bench.py on the CPU: two gloo ranks.

Each rank is an independent replica of the whole workload (no collective on
the data path); the only cross-rank steps are the barriers and the maximum of
the per-rank times, from which the whole-job rate is formed.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slow = bench.max_over_ranks(10.0 + rank, "cpu")          # rank 1 is the slower one
        dist.barrier()
        rate = bench.whole_job_rate(world, 100_000, slow / 1e3)
        q.put((rank, slow, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    assert [g[1] for g in got] == [11.0, 11.0]
    # 2 replicas x 100,000 stamps in 11 ms
    assert all(abs(g[2] - 2 * 100_000 / 0.011) < 1e-3 for g in got)


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_other_ranks_do_no_work():
    class A:
        steps = warmup = 1
        ref_stamps = 10
    assert bench.run_reference(A(), rank=1, world=2) is None

