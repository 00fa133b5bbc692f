"""Ragged batches through size-class launches (fse_fit_batch_ragged), the CUDA
graph replay and the launch-shape autotuner, through the C ABI (needs a GB300).

A stamp's result depends only on its pixels and on how many warps share it
(the summation order).  With one warp per stamp the ragged path must reproduce
fse_fit_batch byte for byte; with the library's or the autotuner's shapes
(several warps on large stamps) it must meet the parity gate against the FP64
oracle, and a captured graph must replay the eager launches byte for byte.
"""
import numpy as np
import pytest
import torch

import parity as PR
from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth

pytestmark = pytest.mark.gpu
ONE = dict(warps_per_stamp=1)


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return B.Context(0)


@pytest.fixture(scope="module")
def ragged():
    cpu = synth.make_workload(2, count=3000)
    b = cpu.to("cuda")
    return cpu, b, B.make_index(b.offset, b.h, b.w)


def single(ctx, b, idx, **kw):
    return ctx.fit_batch(b.pix, idx, scale=b.scale, opts=B.default_opts(max_pix=128 * 128, **ONE, **kw))


def test_ragged_equals_single_launch(ctx, ragged):
    _, b, idx = ragged
    ref = single(ctx, b, idx)
    out = ctx.fit_batch_ragged(b.pix, idx, opts=B.default_opts(**ONE))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # every size class is represented in this sample
    npix = (b.h * b.w).cpu().numpy()
    bounds = [0, 256, 576, 1024, 2304, 4096, 9216, 16384]
    counts = [int(((npix > lo) & (npix <= hi)).sum()) for lo, hi in zip(bounds[:-1], bounds[1:])]
    assert all(c > 0 for c in counts[:-1]), counts


def test_graph_capture_and_replay(ctx, ragged):
    _, b, idx = ragged
    for kw in (ONE, {}):
        ref = ctx.fit_batch_ragged(b.pix, idx, opts=B.default_opts(**kw))          # eager
        opts = B.default_opts(flags=1, **kw)
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


def test_default_and_tuned_shapes_meet_parity(ctx, oracle, ragged):
    cpu, b, idx = ragged
    O = oracle.get()
    ids = np.sort(np.random.default_rng(13).choice(cpu.count, 300, replace=False))
    o = PR.oracle_results(O, cpu, ids)
    default = B.results(ctx.fit_batch_ragged(b.pix, idx))
    rep = PR.compare(default[ids], o, O=O, batch=cpu, ids=ids)
    PR.dump("ragged_default_shapes", rep)
    PR.assert_gate(rep, max_gpu_short=3, max_subpixel=3)
    ctx.autotune(b.pix, idx)
    shapes = ctx.tuned_warps()
    assert len(shapes) == 7 and all(c in (1, 2, 4, 8) and n in (1, 2, 4, 8) and c % n == 0
                                    for c, n in shapes), shapes
    eager = ctx.fit_batch_ragged(b.pix, idx)
    graph = ctx.fit_batch_ragged(b.pix, idx, opts=B.default_opts(flags=1))
    torch.cuda.synchronize()
    assert torch.equal(eager, graph)
    rep = PR.compare(B.results(eager)[ids], o, O=O, batch=cpu, ids=ids)
    PR.dump("ragged_tuned_shapes", rep)
    PR.assert_gate(rep, max_gpu_short=3, max_subpixel=3)


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
        ref = ctx.fit_batch(px, ix, opts=B.default_opts(**ONE))
        out = ctx.fit_batch_ragged(px, ix, opts=B.default_opts(**ONE))
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    r = B.results(ctx.fit_batch_ragged(px, bad))
    assert r["status"][0] == B.ST["BAD_SIZE"] and r["status"][1] == B.ST["BAD_SIZE"]
    # bf16 pixels with per-stamp scales
    bb = synth.encode_bf16(synth.make_workload(2, count=500)).to("cuda")
    ib = B.make_index(bb.offset, bb.h, bb.w)
    ref = single(ctx, bb, ib)
    out = ctx.fit_batch_ragged(bb.pix, ib, scale=bb.scale, opts=B.default_opts(flags=1, **ONE))
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


OTHER_DEVICE = ('{"device": "Some Other GPU", "dtype": "f32", "inv_var": 0, '
                '"class_pix": [256, 576, 1024, 2304, 4096, 9216, 16384], '
                '"warps_per_cta": [1, 1, 1, 1, 1, 1, 1], "warps_per_stamp": [1, 1, 1, 1, 1, 1, 1]}')


def test_tuned_shapes_saved_and_reused_by_a_new_context(ragged, tmp_path):
    """fse_tuning_save / fse_tuning_load: the shapes one context's autotuner
    chose are reused by a new context (another process would do the same)
    without timing again: the same shapes and byte-identical ragged results.
    Entries of other devices in the file are kept; a file with none for this
    device leaves the library's shapes."""
    import json
    cpu, b, idx = ragged
    tuner = B.Context(0)
    tuner.autotune(b.pix, idx)
    shapes = tuner.tuned_warps()
    path = tmp_path / "shapes.json"
    path.write_text('{"format": "libfse-launch-shapes/1", "entries": [\n' + OTHER_DEVICE + '\n]}\n')
    tuner.tuning_save(str(path))
    saved = json.loads(path.read_text())
    assert saved["format"] == "libfse-launch-shapes/1"
    devices = [e["device"] for e in saved["entries"]]
    assert "Some Other GPU" in devices and torch.cuda.get_device_name(0) in devices, devices
    mine = [e for e in saved["entries"] if e["device"] == torch.cuda.get_device_name(0)]
    assert [(c, n) for c, n in zip(mine[0]["warps_per_cta"], mine[0]["warps_per_stamp"])] == shapes

    fresh = B.Context(0)
    assert fresh.tuning_load(str(path))
    assert fresh.tuned_warps() == shapes
    r_tuner = tuner.fit_batch_ragged(b.pix, idx)
    r_fresh = fresh.fit_batch_ragged(b.pix, idx)
    torch.cuda.synchronize()
    assert torch.equal(r_tuner, r_fresh)

    other = tmp_path / "other.json"
    other.write_text('{"format": "libfse-launch-shapes/1", "entries": [\n' + OTHER_DEVICE + '\n]}\n')
    plain = B.Context(0)
    defaults = plain.tuned_warps()
    assert not plain.tuning_load(str(other))
    assert not plain.tuning_load(str(tmp_path / "missing.json"))
    assert plain.tuned_warps() == defaults
