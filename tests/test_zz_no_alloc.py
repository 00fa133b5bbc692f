"""fse_fit_batch_static (scratch in static device memory, no allocation in the
call) against fse_fit_batch, through the C ABI.  The file sorts last so that it
also runs after the other GPU tests; it passes alone in a fresh process too,
where its first call does the per-device setup itself."""
import numpy as np
import pytest
import torch

from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth

pytestmark = pytest.mark.gpu


def test_static_entry_matches_fit_batch():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    batch = synth.make_workload(1, count=4000, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    opts = B.default_opts(max_pix=48 * 48)
    # two calls in a row: the second must find its scratch cleared again
    first = B.results(B.fit_batch_static(batch.pix, idx, opts=opts))
    out = torch.zeros((batch.count, 64), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    B.fit_batch_static(batch.pix, idx, opts=opts, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before    # nothing allocated by the call
    second = B.results(out)
    ref = B.results(B.Context(0).fit_batch(batch.pix, idx, opts=opts))
    assert ((ref["status"] & 3) == 3).mean() > 0.9
    # the same two kernels with the same arguments: the results are identical,
    # byte for byte, on both calls (a scratch word left non-zero by the first
    # call would make the second skip or repeat stamps)
    assert first.tobytes() == ref.tobytes()
    assert second.tobytes() == ref.tobytes()

