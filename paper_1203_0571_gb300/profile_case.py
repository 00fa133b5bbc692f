"""A small, self-contained launch of libfse for profiler captures.

    python -m paper_1203_0571_gb300.profile_case [--what fit_batch|ragged|adjoint|star|moment_vjp|moment_jvp|cutout]
        [--profile gauss|moffat] [--workload 1] [--stamps 20000] [--warmup 3] [--launches 1] [--bf16]

Generates the first `stamps` stamps of a synthetic workload on the GPU, runs
`warmup` launches, then `launches` more, and prints the per-launch time.
fit_batch runs the whole chain; ragged runs fse_fit_batch_ragged on a whole
ragged workload (default the 1,000,000 ragged stamps; --workload 4 the
4,000,000 stamps of 32-64 px, --bf16 with bf16 pixels) after fse_autotune,
as a replayed CUDA graph; adjoint runs fse_sersic_chi2_grad at the
generating parameters with the pixel gradient (the backward launch of the
autograd bridge); star runs fse_star_fit (Sec. 4.2) at the centre and
ellipticity of a preceding fse_centroid + fse_ellipticity; moment_vjp and
moment_jvp run the implicit gradients of that fixed point (sigma_w from the
growth curve), on 100,000 stamps of 48x48 (922 MB read; the VJP writes as
much).  cutout runs fse_cutout on 500 images of 512x512 (524 MB) and then
fse_fit_batch on the cut-outs.  The inputs of the
default cases (20,000 stamps of 48x48 fp32, 184 MB; for the adjoint, 16,384
stamps of 64x64, 268 MB; for the stars, 50,000 Gaussian stars of 32x32, 205
MB, or 50,000 Moffat stars of 48x48, 461 MB) are larger than the 129 MB L2,
so DRAM counters taken on them are meaningful.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import binding as B
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", choices=["fit_batch", "ragged", "adjoint", "star", "moment_vjp", "moment_jvp",
                                       "cutout"],
                    default="fit_batch")
    ap.add_argument("--bf16", action="store_true", help="ragged: pixels stored as bf16 with a per-stamp scale")
    ap.add_argument("--profile", choices=["gauss", "moffat"], default="gauss")
    ap.add_argument("--supersample", type=int, default=1,
                    help="fit_batch: the fit's model as the mean of S x S samples per pixel")
    ap.add_argument("--sigw", choices=["r50", "matched", "fixed"], default="r50",
                    help="sigma_w rule of the implicit gradients (moment_vjp, moment_jvp)")
    ap.add_argument("--workload", type=int, default=None)
    ap.add_argument("--stamps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--launches", type=int, default=1)
    args = ap.parse_args()
    ctx = B.Context(0)
    if args.what == "adjoint":
        return adjoint(ctx, args.workload if args.workload is not None else 3,
                       args.stamps if args.stamps is not None else 16384, args.warmup, args.launches)
    if args.what in ("moment_vjp", "moment_jvp"):
        return moment_grad(ctx, args.what == "moment_jvp", args.workload if args.workload is not None else 1,
                           args.stamps if args.stamps is not None else 100000, args.warmup, args.launches,
                           args.sigw)
    if args.what == "ragged":
        return ragged(ctx, args.workload if args.workload is not None else 2, args.stamps, args.warmup,
                      args.launches, args.bf16)
    if args.what == "cutout":
        return cutout(ctx, args.stamps if args.stamps is not None else 500, args.warmup, args.launches)
    if args.what == "star":
        return star(ctx, args.profile, args.workload if args.workload is not None else
                    (6 if args.profile == "gauss" else 7),
                    args.stamps if args.stamps is not None else 50000, args.warmup, args.launches)
    batch = synth.make_workload(args.workload if args.workload is not None else 1,
                                count=args.stamps if args.stamps is not None else 20000, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    opts = B.default_opts(max_pix=int((batch.h.long() * batch.w.long()).max()), supersample=args.supersample)
    out = torch.empty((batch.count, 64), dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.fit_batch(batch.pix, idx, out=out, opts=opts)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.launches):
        ctx.fit_batch(batch.pix, idx, out=out, opts=opts)
    b.record()
    ctx.sync_check()
    res = B.results(out)
    print(json.dumps({"stamps": batch.count, "ms_per_launch": a.elapsed_time(b) / args.launches,
                      "converged": float(((res["status"] & 3) == 3).mean()),
                      "it_mom": float(res["it_mom"].mean()), "it_fit": float(res["it_fit"].mean())}))


def adjoint(ctx, workload, stamps, warmup, launches):
    import numpy as np
    batch = synth.make_workload(workload, count=stamps, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    t = batch.truth
    p = torch.as_tensor(np.stack([t["xc"], t["yc"], t["g1"], t["g2"], t["I0"], t["re"], t["n"]], axis=1)
                        .astype(np.float32)).cuda()
    gout = torch.ones(batch.count, dtype=torch.float64, device="cuda")
    kw = dict(gout=gout, want_chi2=False, want_dpix=True)
    for _ in range(warmup):
        ctx.chi2_grad(batch.pix, idx, p, **kw)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(launches):
        ctx.chi2_grad(batch.pix, idx, p, **kw)
    b.record()
    ctx.sync_check()
    print(json.dumps({"stamps": batch.count, "pixels": batch.pix.numel(),
                      "ms_per_launch": a.elapsed_time(b) / launches}))


def star(ctx, profile, workload, stamps, warmup, launches):
    batch = synth.make_workload(workload, count=stamps, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    opts = B.default_opts(max_pix=int((batch.h.long() * batch.w.long()).max()))
    mom = ctx.centroid(batch.pix, idx, opts=opts)
    ctx.ellipticity(batch.pix, idx, mom, opts=opts)
    out = torch.empty((batch.count, 32), dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        ctx.star_fit(batch.pix, idx, mom, profile=profile, opts=opts, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(launches):
        ctx.star_fit(batch.pix, idx, mom, profile=profile, opts=opts, out=out)
    b.record()
    ctx.sync_check()
    r = B.star_results(out)
    conv = (r["status"] & 1) == 1
    print(json.dumps({"stamps": batch.count, "pixels": batch.pix.numel(), "profile": profile,
                      "ms_per_launch": a.elapsed_time(b) / launches, "converged": float(conv.mean()),
                      "passes": int(r["iters"][conv].sum()), "passes_mean": float(r["iters"][conv].mean())}))


def moment_grad(ctx, jvp, workload, stamps, warmup, launches, sigw):
    batch = synth.make_workload(workload, count=stamps, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    opts = B.default_opts(max_pix=int((batch.h.long() * batch.w.long()).max()),
                          sigw_mode=1 if sigw == "r50" else 0)
    mode = B.FSE_MOM_ELLIP | {"r50": B.FSE_MOM_SIGW_R50, "matched": 0, "fixed": B.FSE_MOM_SIGW_FIXED}[sigw]
    mom = ctx.centroid(batch.pix, idx, opts=opts)
    ctx.ellipticity(batch.pix, idx, mom, opts=opts)
    g = torch.Generator(device="cuda").manual_seed(1)
    st = torch.zeros(batch.count, dtype=torch.int32, device="cuda")
    if jvp:
        arg = torch.randn(batch.pix.numel(), generator=g, device="cuda")
        out = torch.empty((batch.count, 5), dtype=torch.float32, device="cuda")
        call = lambda: ctx.moment_jvp(batch.pix, idx, mom, arg, out=out, status=st, mode=mode)
    else:
        arg = torch.randn((batch.count, 5), generator=g, device="cuda")
        out = torch.empty(batch.pix.numel(), dtype=torch.float32, device="cuda")
        call = lambda: ctx.moment_vjp(batch.pix, idx, mom, arg, out=out, status=st, mode=mode)
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(launches):
        call()
    b.record()
    ctx.sync_check()
    print(json.dumps({"stamps": batch.count, "pixels": batch.pix.numel(), "what": "jvp" if jvp else "vjp",
                      "sigw": sigw,
                      "ms_per_launch": a.elapsed_time(b) / launches,
                      "status_zero": float((st == 0).float().mean())}))


def ragged(ctx, workload, stamps, warmup, launches, bf16):
    """fse_fit_batch_ragged on a whole ragged workload: autotuned launch shapes,
    captured once into a CUDA graph and replayed."""
    import time
    batch = synth.make_workload(workload, count=stamps, device="cuda")
    if bf16:
        batch = synth.encode_bf16(batch)
    idx = B.make_index(batch.offset, batch.h, batch.w)
    out = torch.empty((batch.count, 64), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.autotune(batch.pix, idx, scale=batch.scale, out=out)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t
    gopts = B.default_opts(flags=B.FSE_FLAG_GRAPH)
    for _ in range(max(warmup, 1)):      # the first call captures the graph
        ctx.fit_batch_ragged(batch.pix, idx, scale=batch.scale, out=out, opts=gopts)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(launches):
        ctx.fit_batch_ragged(batch.pix, idx, scale=batch.scale, out=out, opts=gopts)
    b.record()
    ctx.sync_check()
    ms = a.elapsed_time(b) / launches
    res = B.results(out)
    npx = float((batch.h.long() * batch.w.long()).sum())
    print(json.dumps({"workload": synth.WORKLOADS[workload].name, "stamps": batch.count, "pixels": npx,
                      "pixel_dtype": "bf16" if bf16 else "f32", "ms_per_call": ms,
                      "stamps_per_s": batch.count / (ms / 1e3), "pixels_per_s": npx / (ms / 1e3),
                      "tune_s": tune_s, "tuned_warps": ctx.tuned_warps(B.FSE_BF16 if bf16 else B.FSE_F32),
                      "converged": float(((res["status"] & 3) == 3).mean())}))


def cutout(ctx, images, warmup, launches):
    batch = synth.make_workload(8, count=images, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    pix, cidx, info = ctx.cutout(batch.pix, idx)
    opts = B.default_opts(max_pix=128 * 128)
    out = torch.empty((batch.count, 64), dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        ctx.cutout(batch.pix, idx, out=pix)
        ctx.fit_batch(pix, cidx, opts=opts, out=out)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(launches):
        ctx.cutout(batch.pix, idx, out=pix)
    ev[1].record()
    for _ in range(launches):
        ctx.fit_batch(pix, cidx, opts=opts, out=out)
    ev[2].record()
    ctx.sync_check()
    inf = B.cutout_info(info)
    res = B.results(out)
    print(json.dumps({"images": batch.count, "image_pixels": batch.pix.numel(), "cutout_pixels": pix.numel(),
                      "side_median": float(np.median(inf["h"])),
                      "ms_cutout": ev[0].elapsed_time(ev[1]) / launches,
                      "ms_fit_batch": ev[1].elapsed_time(ev[2]) / launches,
                      "converged": float(((res["status"] & 3) == 3).mean())}))


if __name__ == "__main__":
    main()
