"""A small, self-contained launch of fse_fit_batch for profiler captures.

    python -m paper_1203_0571_gb300.profile_case [--workload 1] [--stamps 20000]
                                                 [--warmup 3] [--launches 1]

Generates the first `stamps` stamps of a synthetic workload on the GPU, runs
`warmup` launches, then `launches` more, and prints the per-launch time.  The
inputs of the default case (20,000 stamps of 48x48 fp32, 184 MB) are larger
than the 129 MB L2, so DRAM counters taken on it are meaningful.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from . import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--stamps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--launches", type=int, default=1)
    args = ap.parse_args()
    ctx = B.Context(0)
    batch = synth.make_workload(args.workload, count=args.stamps, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    opts = B.default_opts(max_pix=int((batch.h.long() * batch.w.long()).max()))
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


if __name__ == "__main__":
    main()
