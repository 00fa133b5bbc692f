"""Per-parameter error of the CUDA path against the FP64 oracle on the
low-SNR precision subsample, with fp32 and bf16 pixel storage.

    python tests/precision_report.py [--stamps 10000] [--markdown out.md]

The subsample is the precision-lowsnr workload: side ~ U{32..64}, SNR ~
U[10, 30], n ~ U[0.5, 8].  The GPU runs the whole chain (fse_fit_batch_ragged)
on the fp32 pixels and on the same pixels stored as bf16 with one scale per
stamp (scale = max |I|).  Errors are reported three ways:

  fp32        GPU on fp32 pixels        vs the oracle on the fp32 pixels
  bf16 comp.  GPU on bf16 pixels        vs the oracle on the decoded bf16 pixels
                                           (the arithmetic alone)
  bf16 total  GPU on bf16 pixels        vs the oracle on the fp32 pixels
                                           (storage plus arithmetic)

Stamps enter a comparison as in the parity gate: both sides converged,
neither fit ended on a bound, the oracle's J^T J is not degenerate
(condition number <= 1e10) and the GPU did not find another, lower minimum.  For each parameter the report gives the
median, the 99th percentile and the maximum error (absolute for x0, y0, e1,
e2; relative for r_e, n, flux, chi^2) and the fraction within the parity
tolerance.  It also gives the median statistical error of each parameter
(from the oracle's J^T J at its optimum, for r_e and n), so that a storage
error can be read against the noise.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import parity as PR  # noqa: E402

KEYS = ("x0", "y0", "e1", "e2", "re", "n", "flux", "chi2")


def gpu_results(batch, count):
    import torch
    from paper_1203_0571_gb300 import binding as B
    ctx = B.Context(0)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    out = ctx.fit_batch_ragged(b.pix, idx, scale=b.scale)
    torch.cuda.synchronize()
    return B.results(out)


def errors(g, o, O, batch, same_pixels=True):
    # on different pixels (storage error) chi^2 values are not comparable, and
    # neither is the "lower chi^2 means another basin" exclusion built on them
    keys = KEYS if same_pixels else tuple(k for k in KEYS if k != "chi2")
    rep = PR.compare(g, o, keys=keys, O=O, batch=batch, ids=np.arange(batch.count), same_pixels=same_pixels)
    gate = rep["_gate"]
    row = {"gated": int(gate.sum()), "total": int(gate.size), "reasons": dict(rep["reasons"]),
           "excluded": {k: rep[k] for k in ("excluded_condition", "excluded_other_minimum",
                                             "excluded_clamped_fixed_point", "excluded_other_fixed_point",
                                             "gpu_short", "subpixel", "unconfirmed")}}
    for k in keys:
        e = rep["_err"][k][gate]
        row[k] = {"median": float(np.median(e)) if e.size else 0.0,
                  "p99": float(np.percentile(e, 99)) if e.size else 0.0,
                  "max": float(e.max()) if e.size else 0.0,
                  "within": float(np.mean(e <= PR.TOL[k])) if e.size else 1.0}
    return row


def stat_errors(O, batch, o):
    """Median 1-sigma errors of r_e and n (relative) from the oracle's J^T J."""
    sr, sn = [], []
    for i in range(len(o)):
        r = o[i]
        if (r["status"] & 3) != 3 or r["status"] & 128:
            continue
        _, _, H = O.fit_eval(batch.stamp(i), r["x0"], r["y0"], r["e1"], r["e2"], [r["I0"], r["re"], r["n"]])
        try:
            C = np.linalg.inv(H)
        except np.linalg.LinAlgError:
            continue
        if C[1, 1] > 0 and C[2, 2] > 0:
            sr.append(np.sqrt(C[1, 1]) / r["re"])
            sn.append(np.sqrt(C[2, 2]) / r["n"])
    return {"re": float(np.median(sr)) if sr else float("nan"),
            "n": float(np.median(sn)) if sn else float("nan")}


def run(stamps: int):
    import oracle
    from paper_1203_0571_gb300 import synth
    O = oracle.get()
    f32 = synth.make_workload(5, count=stamps)
    b16 = synth.encode_bf16(f32)
    ids = np.arange(stamps)
    o32 = PR.oracle_results(O, f32, ids)
    o16 = PR.oracle_results(O, b16, ids)
    g32 = gpu_results(f32, stamps)
    g16 = gpu_results(b16, stamps)
    report = {"stamps": stamps, "workload": "precision-lowsnr (side U{32..64}, SNR U[10,30], n U[0.5,8])",
              "fp32": errors(g32, o32, O, f32), "bf16_compute": errors(g16, o16, O, b16),
              "bf16_total": errors(g16, o32, O, f32, same_pixels=False),
              "oracle_sigma_median": stat_errors(O, f32, o32[:min(stamps, 2000)])}
    return report


def markdown(rep) -> str:
    lines = [f"Workload: {rep['workload']}, {rep['stamps']} stamps.", "",
             "| comparison | gated | " + " | ".join(KEYS) + " |",
             "|---|---|" + "---|" * len(KEYS)]
    for name, lab in (("fp32", "fp32 pixels vs oracle"), ("bf16_compute", "bf16: arithmetic (oracle on decoded bf16)"),
                      ("bf16_total", "bf16: storage + arithmetic (oracle on fp32)")):
        r = rep[name]
        for stat in ("median", "p99", "max", "within"):
            cells = [("—" if k not in r else f"{r[k][stat]:.1%}" if stat == "within" else f"{r[k][stat]:.1e}")
                     for k in KEYS]
            lines.append(f"| {lab} — {stat} | {r['gated']}/{r['total']} | " + " | ".join(cells) + " |")
    s = rep["oracle_sigma_median"]
    lines += ["", f"Median 1-sigma statistical error (oracle J^T J): r_e {s['re']:.1e} relative, n {s['n']:.1e} relative."]
    for name in ("fp32", "bf16_compute"):
        ex = rep[name]["reasons"]
        lines.append(f"Outside the gate ({name}), by reason: " +
                     (", ".join(f"{k} {v}" for k, v in sorted(ex.items())) or "none") + ".")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--stamps", type=int, default=10000)
    ap.add_argument("--markdown", default=None)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    rep = run(args.stamps)
    md = markdown(rep)
    print(md)
    if args.markdown:
        with open(args.markdown, "w") as f:
            f.write(md + "\n")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
