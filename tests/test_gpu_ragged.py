"""Ragged batches through size-class launches (fse_fit_batch_ragged), the CUDA
graph replay and the launch-shape autotuner, through the C ABI (needs a GB300).

Each stamp is measured on its own by one warp, so its result cannot depend
on which launch, tile size or launch shape processed it: the ragged path must
reproduce fse_fit_batch byte for byte.  fse_fit_batch itself is held to the
FP64 oracle by the parity tests.
"""
import numpy as np
import pytest
import torch

from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return B.Context(0)


@pytest.fixture(scope="module")
def ragged():
    b = synth.make_workload(2, count=3000).to("cuda")
    return b, B.make_index(b.offset, b.h, b.w)


def reference(ctx, b, idx):
    return ctx.fit_batch(b.pix, idx, opts=B.default_opts(max_pix=128 * 128))


def test_ragged_equals_single_launch(ctx, ragged):
    b, idx = ragged
    ref = reference(ctx, b, idx)
    out = ctx.fit_batch_ragged(b.pix, idx)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # every size class is represented in this sample
    npix = (b.h * b.w).cpu().numpy()
    bounds = [0, 256, 576, 1024, 2304, 4096, 9216, 16384]
    counts = [int(((npix > lo) & (npix <= hi)).sum()) for lo, hi in zip(bounds[:-1], bounds[1:])]
    assert all(c > 0 for c in counts[:-1]), counts


def test_graph_capture_and_replay(ctx, ragged):
    b, idx = ragged
    ref = reference(ctx, b, idx)
    opts = B.default_opts(flags=1)
    out = torch.zeros_like(ref)
    ctx.fit_batch_ragged(b.pix, idx, opts=opts, out=out)      # captures
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    out.zero_()
    ctx.fit_batch_ragged(b.pix, idx, opts=opts, out=out)      # replays
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    other = torch.zeros_like(ref)                             # new pointer: captures again
    ctx.fit_batch_ragged(b.pix, idx, opts=opts, out=other)
    torch.cuda.synchronize()
    assert torch.equal(other, ref)


def test_autotune_keeps_results(ctx, ragged):
    b, idx = ragged
    ref = reference(ctx, b, idx)
    out = ctx.autotune(b.pix, idx)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    w = ctx.tuned_warps()
    assert len(w) == 7 and all(x in (1, 2, 4, 8) for x in w), w
    out2 = ctx.fit_batch_ragged(b.pix, idx, opts=B.default_opts(flags=1))
    torch.cuda.synchronize()
    assert torch.equal(out2, ref)


def test_ragged_with_invalid_sizes_and_bf16(ctx):
    rng = np.random.default_rng(5)
    stamps = [rng.normal(size=(h, w)) + 2.0 for h, w in ((20, 20), (129, 129), (40, 33), (1, 1))]
    stamps.append(synth.single_stamp(70, 66, n=2.0, re=6.0, g1=0.1, g2=-0.2, xc=32.4, yc=35.1,
                                     I0=300.0, noise_sigma=1.0, seed=3))
    pix = np.concatenate([s.astype(np.float32).ravel() for s in stamps])
    offs = np.cumsum([0] + [s.size for s in stamps[:-1]])
    idx = B.make_index(offs, [s.shape[0] for s in stamps], [s.shape[1] for s in stamps])
    # the same buffer with the first stamp's height set to 0 (an empty stamp)
    bad = B.make_index(offs, [0, 129, 40, 1, 70], [5, 129, 33, 1, 66])
    px = torch.as_tensor(pix).cuda()
    for ix in (idx, bad):
        ref = ctx.fit_batch(px, ix)
        out = ctx.fit_batch_ragged(px, ix)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    r = B.results(ctx.fit_batch_ragged(px, bad))
    assert r["status"][0] == B.ST["BAD_SIZE"] and r["status"][1] == B.ST["BAD_SIZE"]
    # bf16 pixels with per-stamp scales
    bb = synth.encode_bf16(synth.make_workload(2, count=500)).to("cuda")
    ib = B.make_index(bb.offset, bb.h, bb.w)
    ref = ctx.fit_batch(bb.pix, ib, scale=bb.scale)
    out = ctx.fit_batch_ragged(bb.pix, ib, scale=bb.scale, opts=B.default_opts(flags=1))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
