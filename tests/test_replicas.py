"""Replicas over stamp ranges (CPU): fse_partition's boundaries, and the
split -> per-rank work -> gather -> concatenation with two gloo ranks, where
each rank runs the FP64 oracle on its range and rank 0 must get the one-call
result back in order."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1203_0571_gb300 import binding as B  # noqa: E402


def _px(h, w):
    ok = (h >= 1) & (w >= 1) & (h <= 128) & (w <= 128)
    return np.where(ok, h.astype(np.int64) * w, 1)


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 64])
def test_partition_ranges_are_contiguous_and_balanced(parts):
    rng = np.random.default_rng(parts)
    n = 5000
    h = rng.integers(16, 129, n)
    w = h.copy()
    h[::97] = 0                                   # invalid sizes weigh one pixel
    idx = B.make_index(np.arange(n) * 7, h, w, device="cpu")
    s = B.partition(idx, parts)
    assert s[0] == 0 and s[-1] == n and np.all(np.diff(s) >= 0) and len(s) == parts + 1
    px = _px(h, w)
    cum = np.concatenate([[0], np.cumsum(px)])
    share = cum[-1] / parts
    for r in range(parts):
        got = cum[s[r + 1]] - cum[s[r]]
        assert abs(got - share) <= px.max() + 1, (r, got, share)
        # range r starts at the first stamp at or past r/parts of the pixels
        if 0 < r:
            assert cum[s[r]] >= r * share - 1e-6 and (s[r] == 0 or cum[s[r] - 1] < r * share), r


def test_partition_edge_cases():
    idx = B.make_index([0, 10], [2, 3], [5, 4], device="cpu")
    # 10 and 12 pixels: range r starts at the first stamp at or past 22 r / 5 pixels
    assert list(B.partition(idx, 5)) == [0, 1, 1, 2, 2, 2]
    assert list(B.partition(idx, 1)) == [0, 2]
    empty = B.make_index([], [], [], device="cpu")
    assert list(B.partition(empty, 3)) == [0, 0, 0, 0]
    with pytest.raises(B.FseError):
        B.partition(idx, 0)


def _port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1203_0571_gb300 import replicas, synth
        batch = synth.make_workload(2, count=40)           # ragged sizes: unequal ranges
        idx = B.make_index(batch.offset, batch.h, batch.w, device="cpu")
        starts = B.partition(idx, world)
        a, b = replicas.rank_range(starts, rank)
        O = oracle.get()
        res, _ = O.batch(batch.pix.numpy(), batch.offset.numpy()[a:b], batch.h.numpy()[a:b],
                         batch.w.numpy()[a:b], threads=1)
        rec = torch.as_tensor(res.view(np.uint8).reshape(b - a, -1).copy())
        full = replicas.gather_records(rec, starts)
        if rank == 0:
            one, _ = O.batch(batch.pix.numpy(), batch.offset.numpy(), batch.h.numpy(), batch.w.numpy(),
                             threads=1)
            q.put((rank, full.numpy().tobytes() == one.view(np.uint8).tobytes(), list(starts)))
        else:
            q.put((rank, full is None, list(starts)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_and_concatenate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    assert got[0][1] and got[1][1], got
    assert got[0][2] == got[1][2] and 0 < got[0][2][1] < 40
