"""Replicas over stamp ranges on one GPU: the ranges of fse_partition fitted
one after another, each by its own fse_fit_batch call, and concatenated in
range order equal one fse_fit_batch call over the whole batch byte for byte
(every stamp is independent, and one warp per stamp sums in a fixed order)."""
import numpy as np
import pytest
import torch

from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import replicas, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("parts", [2, 3, 8])
def test_ranges_concatenate_to_the_one_call_result(parts):
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    ctx = B.Context(0)
    batch = synth.make_workload(2, count=4000)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    opts = B.default_opts(max_pix=128 * 128, warps_per_stamp=1)
    one = ctx.fit_batch(b.pix, idx, opts=opts)
    starts = B.partition(idx.cpu(), parts)
    pieces = [replicas.fit_range(ctx, b.pix, idx, starts, r, opts=opts) for r in range(parts)]
    torch.cuda.synchronize()
    assert sum(p.shape[0] for p in pieces) == batch.count
    assert torch.equal(torch.cat(pieces), one)
    px = (batch.h.long() * batch.w.long()).numpy()
    shares = [px[starts[r]:starts[r + 1]].sum() for r in range(parts)]
    assert max(shares) - min(shares) <= 2 * px.max()
