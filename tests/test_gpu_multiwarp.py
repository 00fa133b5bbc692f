"""Several warps per stamp (fse_opts.warps_per_stamp) against the FP64 oracle,
through the C ABI (needs a GB300).  The summation order differs from one warp
per stamp, so the comparison is the parity gate, not bit equality."""
import numpy as np
import pytest
import torch

import parity as PR
from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return B.Context(0)


@pytest.fixture(scope="module")
def ragged(oracle):
    batch = synth.make_workload(2, count=1200)
    ids = np.sort(np.random.default_rng(11).choice(batch.count, 240, replace=False))
    return batch, ids, PR.oracle_results(oracle.get(), batch, ids)


@pytest.mark.parametrize("nw", [2, 4, 8])
def test_warps_per_stamp_parity(ctx, oracle, ragged, nw):
    batch, ids, o = ragged
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    g = B.results(ctx.fit_batch(b.pix, idx, opts=B.default_opts(max_pix=128 * 128, warps_per_stamp=nw,
                                                                 warps_per_cta=nw)))
    rep = PR.compare(g[ids], o, O=oracle.get(), batch=batch, ids=ids)
    PR.dump(f"multiwarp_{nw}", rep)
    PR.assert_gate(rep, max_gpu_short=3, max_subpixel=3)


def test_multiwarp_bf16_and_inverse_variance(ctx, oracle):
    O = oracle.get()
    batch = synth.make_workload(3, count=48)
    ivar = (0.5 + np.random.default_rng(12).random(batch.pix.numel())).astype(np.float32)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    ids = np.arange(batch.count)
    g = B.results(ctx.fit_batch(b.pix, idx, inv_var=torch.as_tensor(ivar).cuda(),
                                opts=B.default_opts(max_pix=64 * 64, warps_per_stamp=4, warps_per_cta=8)))
    o = PR.oracle_results(O, batch, ids, ivar=ivar)
    rep = PR.compare(g, o, O=O, batch=batch, ids=ids, ivar=ivar)
    PR.dump("multiwarp_ivar", rep)
    PR.assert_gate(rep, max_gpu_short=1, max_subpixel=1)
    bb = synth.encode_bf16(batch).to("cuda")
    g = B.results(ctx.fit_batch(bb.pix, idx, scale=bb.scale,
                                opts=B.default_opts(max_pix=64 * 64, warps_per_stamp=2, warps_per_cta=4)))
    o = PR.oracle_results(O, synth.encode_bf16(batch), ids)
    rep = PR.compare(g, o, O=O, batch=synth.encode_bf16(batch), ids=ids)
    PR.dump("multiwarp_bf16", rep)
    PR.assert_gate(rep, max_gpu_short=1, max_subpixel=1)


def test_invalid_launch_shapes_are_rejected(ctx):
    b = synth.make_workload(0, count=4).to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    for kw in (dict(warps_per_stamp=3), dict(warps_per_stamp=4, warps_per_cta=2)):
        with pytest.raises(B.FseError):
            ctx.fit_batch(b.pix, idx, opts=B.default_opts(**kw))
    # several warps per stamp only for the whole chain
    with pytest.raises(B.FseError):
        ctx.centroid(b.pix, idx, opts=B.default_opts(warps_per_stamp=2, warps_per_cta=2))
