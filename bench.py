#!/usr/bin/env python3
"""Throughput of the fast shape estimator on GB300.

One step = the whole chain (start-up, centroid + ellipticity, Sérsic fit) over
the uniform 48x48 workload: 100,000 seeded synthetic stamps, fp32 (80% Sérsic
galaxies with SNR U[15,200], 20% Gaussian stars), resident in HBM, in one
persistent launch of fse_fit_batch.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fse|reference]

Under torchrun each rank runs the same workload on its own GPU (independent
replicas, no collective on the data path; weak scaling) and rank 0 prints the
line with the slowest rank's time.  --impl reference times the FP64 CPU oracle
on the host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stamps fitted/sec (centroid+ellipticity+Sérsic fit) at 48×48 fp32; % FP32 roofline"
UNIT = "stamps/s"
WORKLOAD = 1
# Algorithmic fp32 lane-operations per pixel (FMA = 1, MUFU ex2/lg2 = 1) of each
# pass of the method as formulated here; see the design notes for the derivation.
OPS_INIT = 12          # brightest pixel, total, growth-curve ring histogram
OPS_MOMENT = 24        # one weighted pass (11 moments, 1 ex2)
OPS_MOM_REFINE = 88    # one moment refinement pass (exact offsets, ~1-ulp exp2, double-float sums)
OPS_FIT_SETUP = 8 + 26  # 0.5 log2 R^2 per pixel + the four-candidate start pass (8 ex2)
OPS_FIT = 18           # one profile pass (10 sums, 2 ex2)
OPS_REFINE = 76        # one fit refinement pass (two ~1-ulp exp2, double-float and curvature sums)
SMS = 152
LANES_PER_SM = 128


def config_dict(n, world):
    return {
        "workload": "uniform-48px: 100,000 stamps 48x48 fp32, 80% Sersic galaxies "
                    "(n U[0.5,4], r_e U[1.5,5] px, |g| U[0,0.5], SNR U[15,200]), "
                    "20% Gaussian stars (FWHM U[2,4] px, |g|<0.05), noise sigma 1, seed 1",
        "stamps_per_gpu": n,
        "stamp_px": [48, 48],
        "pixel_dtype": "f32",
        "launch": "one fse_fit_batch per step (three persistent kernel launches: start-up, moments, fit)",
        "l2": "inputs 0.92 GB per GPU, larger than the 129 MB L2; no flush",
        "parallelism": f"replicas{world}",
    }


def algorithmic_ops(res) -> float:
    st = res["status"]
    npix = res["npix"].astype(np.float64)
    ok = (st & (32 | 16)) == 0
    fit = ((st & 1) != 0) & ok
    ops = npix * (OPS_INIT + OPS_MOMENT * res["it_mom"]) * ok
    # one refinement pass of each kind, and a second where the status says it ran
    ops += npix * OPS_MOM_REFINE * (1 + ((st & (1 << 13)) != 0)) * fit
    ops += npix * (OPS_FIT_SETUP + OPS_FIT * res["it_fit"]) * fit
    ops += npix * OPS_REFINE * (1 + ((st & (1 << 14)) != 0)) * (((st & 2) != 0) & ((st & 128) == 0) & fit)
    return float(ops.sum())


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.device)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.25)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        pw = [num(r[3]) for r in rows if num(r[3])]
        busy = [num(r[1]) for r in rows if num(r[3]) and num(r[3]) > 0.5 * max(pw)] if pw else sm
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6),
                              ("sw_thermal_slowdown", 7), ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(busy or sm), "sm_max_mhz": num(rows[0][2]),
                "samples": len(rows), "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons)}


def kernel_traffic():
    """DRAM bytes per launch of the estimator kernel from a committed ncu summary,
    valid only while the kernel source is the one that was profiled."""
    p = os.path.join(ROOT, "profiles", "estimator_traffic.json")
    src = os.path.join(ROOT, "paper_1203_0571_gb300", "csrc", "fse_kernels.cu")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return d.get("dram_bytes_per_launch") if d.get("kernel_sha256") == h else None


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the process group (x itself alone)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, slowest_s: float) -> float:
    """Units per second of the whole job: every rank (a replica) processes
    units_per_rank, and the job ends with the slowest rank."""
    return world * units_per_rank / slowest_s


def cpu_oracle_rate(batch, target_s: float, max_stamps: int):
    """The FP64 oracle on the host cores over a bounded sample of the workload."""
    import oracle as O
    from paper_1203_0571_gb300 import synth
    O.build()
    pilot = 256
    sub = synth.make_workload(WORKLOAD, count=pilot)
    t = time.perf_counter()
    O.batch(sub.pix.numpy(), sub.offset.numpy(), sub.h.numpy(), sub.w.numpy())
    dt = max(time.perf_counter() - t, 1e-3)
    count = int(min(max_stamps, max(pilot, pilot * target_s / dt)))
    sub = synth.make_workload(WORKLOAD, count=count)
    t = time.perf_counter()
    res, used = O.batch(sub.pix.numpy(), sub.offset.numpy(), sub.h.numpy(), sub.w.numpy())
    dt = time.perf_counter() - t
    return {"value": count / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"first {count} stamps of the 100,000-stamp uniform-48px workload, "
                      f"whole chain, FP64, {used} threads, {dt:.2f} s wall",
            "it_mom_mean": float(np.mean(res["it_mom"])), "it_fit_mean": float(np.mean(res["it_fit"]))}


def run_reference(args, rank, world):
    """The oracle as the reference arm, timed on the host cores."""
    if rank != 0:
        return
    import oracle as O
    from paper_1203_0571_gb300 import synth
    O.build()
    per_step = args.ref_stamps
    sub = synth.make_workload(WORKLOAD, count=per_step)
    arrs = (sub.pix.numpy(), sub.offset.numpy(), sub.h.numpy(), sub.w.numpy())
    used = 1
    for _ in range(args.warmup):
        _, used = O.batch(*arrs)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        _, used = O.batch(*arrs)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(100_000, world), reference_sample_per_step=per_step),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"first {per_step} stamps of the uniform-48px workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fse", choices=["fse", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--plain-stamps", type=int, default=10000)
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--ref-stamps", type=int, default=2000)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if args.impl == "reference":
        return run_reference(args, rank, world)

    torch.cuda.set_device(local)
    if dist:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1203_0571_gb300 import binding as B
    from paper_1203_0571_gb300 import synth

    ctx = B.Context(local)
    batch = synth.make_workload(WORKLOAD, device=f"cuda:{local}")
    n = batch.count
    idx = B.make_index(batch.offset, batch.h, batch.w, device=f"cuda:{local}")
    out = torch.empty((n, 64), dtype=torch.uint8, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    opts = B.default_opts(max_pix=48 * 48)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        ctx.fit_batch(batch.pix, idx, out=out, opts=opts, stream=stream)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for a, b in ev:
        a.record(stream)
        ctx.fit_batch(batch.pix, idx, out=out, opts=opts, stream=stream)
        b.record(stream)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = t0.elapsed_time(t1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(total_ms / args.steps, f"cuda:{local}")
    res = B.results(out)
    ops = algorithmic_ops(res)
    kernel_ms = statistics.mean(step_ms)
    peak_gops = SMS * LANES_PER_SM * 2070.0 * 1e6 / 1e9     # at the maximum SM clock
    achieved = ops / (kernel_ms / 1e3) / 1e9
    value = whole_job_rate(world, n, ms / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    host_pix = batch.pix.cpu().pin_memory()
    host_idx = idx.cpu().pin_memory()
    host_out = torch.empty((n, 64), dtype=torch.uint8).pin_memory()
    ctx.fit_batch_host(host_pix, host_idx, out=host_out)
    barrier()
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.fit_batch_host(host_pix, host_idx, out=host_out)
    e2e_s = max_over_ranks((time.perf_counter() - t) / args.e2e_steps, f"cuda:{local}")
    e2e = {"value": whole_job_rate(world, n, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(host_pix.numel() * 4 + host_idx.numel() * 8),
           "d2h_bytes_per_step": int(n * 64), "entry": "fse_fit_batch_host", "ms_per_step": 1e3 * e2e_s}
    same = bool(np.array_equal(host_out.numpy(), out.cpu().numpy()))

    # the plain form: one launch pair per stamp, on the first stamps of the workload
    pn = min(args.plain_stamps, n)
    pout = torch.empty((pn, 64), dtype=torch.uint8, device=f"cuda:{local}")
    ctx.fit_batch_plain(batch.pix, idx[:pn], out=pout, opts=opts)
    torch.cuda.synchronize()
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pa.record(stream)
    ctx.fit_batch_plain(batch.pix, idx[:pn], out=pout, opts=opts, stream=stream)
    pb.record(stream)
    torch.cuda.synchronize()
    plain = {"value": pn / (pa.elapsed_time(pb) / 1e3), "unit": UNIT, "stamps": pn,
             "launches": 3 * pn, "identical_results": bool(torch.equal(pout, out[:pn]))}

    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(batch, args.cpu_seconds, 40000)
    conv = (res["status"] & 3) == 3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(n, world),
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": kernel_traffic(),
                     "kernel": "estimator_kernel<moments> + estimator_kernel<fit> (the two launches of "
                               "one fse_fit_batch, f32)", "kernel_ms": kernel_ms,
                     "ops_per_launch": ops,
                     "peak_source": "152 SMs x 128 fp32 lanes x 2070 MHz (issue slots, FMA = 1 op)"},
        "cpu_baseline": cpu,
        "plain_per_stamp_launch": plain,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
        "stats": {"converged_frac": float(conv.mean()), "it_mom_mean": float(res["it_mom"].mean()),
                  "it_fit_mean": float(res["it_fit"][conv].mean()) if conv.any() else 0.0,
                  "e2e_matches_device": same},
    }
    print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
