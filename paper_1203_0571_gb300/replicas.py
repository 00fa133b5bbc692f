"""Replicas over stamp ranges: one batch spread over the ranks of a process
group (one GPU each).

The stamps are independent, so there is no collective on the data path: the
index is cut into contiguous ranges of about equal total pixels
(fse_partition), every rank fits its own range with fse_fit_batch, and the
result records are concatenated on the host in range order.  The only
cross-rank step is that final gather of the 64-byte records.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def rank_range(starts: np.ndarray, rank: int) -> tuple[int, int]:
    """[start, stop) of this rank's stamps."""
    return int(starts[rank]), int(starts[rank + 1])


def fit_range(ctx: "B.Context", pix: torch.Tensor, index: torch.Tensor, starts: np.ndarray, rank: int,
              **kw) -> torch.Tensor:
    """fse_fit_batch on this rank's stamps (index on the rank's device);
    returns their records (uint8 [n_r, 64]) on that device."""
    a, b = rank_range(starts, rank)
    if b == a:
        return torch.empty((0, 64), dtype=torch.uint8, device=index.device)
    return ctx.fit_batch(pix, index[a:b].contiguous(), **kw)


def gather_records(local: torch.Tensor, starts: np.ndarray, group=None) -> torch.Tensor | None:
    """The records of all ranks, concatenated in range order on rank 0 (host
    memory); None on the other ranks.  local: this rank's records
    (uint8 [n_r, 64], any device)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sizes = [int(starts[r + 1] - starts[r]) for r in range(world)]
    width = local.shape[1] if local.dim() == 2 else 64
    pad = max(sizes) if sizes else 0
    buf = torch.zeros((pad, width), dtype=torch.uint8)
    if local.numel():
        buf[: local.shape[0]] = local.detach().cpu()
    parts = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, gather_list=parts, dst=0, group=group)
    if rank != 0:
        return None
    return torch.cat([parts[r][: sizes[r]] for r in range(world)], dim=0)
