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
OPS_MOMENT = 24        # one weighted pass with the fourth moments (11 sums, 1 ex2)
OPS_MOMENT_2 = 17      # one weighted pass without them (6 sums), counted from the third pass on
OPS_MOM_REFINE = 110   # one moment refinement pass (exact offsets, float-pair weight exponent,
                       # ~1-ulp exp2, double-float sums with the products' rounding kept)
OPS_FIT_SETUP = 8 + 26  # 0.5 log2 R^2 per pixel + the four-candidate start pass (8 ex2)
OPS_FIT = 18           # one profile pass (10 sums, 2 ex2)
OPS_REFINE = 61        # one fit refinement pass (two ~1-ulp exp2, double-float gradient and chi^2
                       # sums, fp32 J^T J and curvature sums)
# The nominal per-pass figures (the "frac_survey" accounting): a moment pass
# 1 ex2 + ~30 fp32 operations, a fit pass 3 MUFU + ~30; every pixel pass the
# kernels run counts once at these rates over the whole stamp (the start-up
# and the refinement passes included, the four-candidate fit start as one fit
# pass).
NOMINAL_MOMENT = 31
NOMINAL_FIT = 33
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


def pass_counts(res):
    """Pixel passes each stamp ran, by kind: start-up, moment iterations (the
    first two with fourth moments), moment refinements, fit start, fit
    iterations, fit refinements.  A refinement runs once, and a second time
    where the status bit says so (more than two are not counted: errs low)."""
    st = res["status"]
    ok = (st & (32 | 16)) == 0
    fit = ((st & 1) != 0) & ok
    it = res["it_mom"].astype(np.float64) * ok
    return {"init": ok.astype(np.float64), "mom4": np.minimum(it, 2.0), "mom": np.maximum(it - 2.0, 0.0),
            "mom_refine": (1.0 + ((st & (1 << 13)) != 0)) * fit, "fit_start": fit.astype(np.float64),
            "fit": res["it_fit"].astype(np.float64) * fit,
            "fit_refine": (1.0 + ((st & (1 << 14)) != 0)) * (((st & 2) != 0) & ((st & 128) == 0) & fit)}


WEIGHT_CUT = 7.4446500   # sqrt(80 ln 2): the moment passes skip pixels with weight below 2^-40


def box_pixels(res, h: int, w: int) -> np.ndarray:
    """Pixels of each stamp's moment box (the bounding box of the weight's
    ellipse R^2 <= 80 ln 2 s_w^2 plus a pixel, cut to the stamp) at the final
    centre, g and s_w; the passes before the last ran on boxes about this
    size.  Stamps without a moment result count the whole stamp."""
    g1 = res["e1"].astype(np.float64)
    g2 = res["e2"].astype(np.float64)
    gg = g1 * g1 + g2 * g2
    with np.errstate(invalid="ignore", divide="ignore"):
        rc = WEIGHT_CUT * res["sigma_w"] / (1.0 - gg)
        hx = np.minimum(rc * np.sqrt(np.maximum(1 + gg + 2 * g1, 0)) + 1, 4096)
        hy = np.minimum(rc * np.sqrt(np.maximum(1 + gg - 2 * g1, 0)) + 1, 4096)
        c0 = np.maximum(0, np.floor(res["x0"] - hx))
        r0 = np.maximum(0, np.floor(res["y0"] - hy))
        c1 = np.minimum(w - 1, np.ceil(res["x0"] + hx))
        r1 = np.minimum(h - 1, np.ceil(res["y0"] + hy))
        n = (c1 - c0 + 1) * (r1 - r0 + 1)
    ok = np.isfinite(n) & (c1 >= c0) & (r1 >= r0)
    return np.where(ok, n, h * w).astype(np.float64)


def algorithmic_ops(res, h: int = 48, w: int = 48) -> float:
    """The builder's count: each pass at the operations it performs per pixel,
    over the pixels it visits (the moment passes over the weight's box)."""
    c = pass_counts(res)
    npix = res["npix"].astype(np.float64)
    nbox = np.minimum(box_pixels(res, h, w), npix)
    ops = (npix * (OPS_INIT * c["init"] + OPS_FIT_SETUP * c["fit_start"] + OPS_FIT * c["fit"] +
                   OPS_REFINE * c["fit_refine"]) +
           nbox * (OPS_MOMENT * c["mom4"] + OPS_MOMENT_2 * c["mom"] + OPS_MOM_REFINE * c["mom_refine"]))
    return float(ops.sum())


def nominal_ops(res) -> float:
    """The nominal count: every pass at 31 (moment kind) or 33 (fit kind) per
    pixel of the whole stamp (the method's nominal work; the kernels visit
    fewer pixels in the moment passes)."""
    c = pass_counts(res)
    per_px = (NOMINAL_MOMENT * (c["init"] + c["mom4"] + c["mom"] + c["mom_refine"]) +
              NOMINAL_FIT * (c["fit_start"] + c["fit"] + c["fit_refine"]))
    return float((res["npix"].astype(np.float64) * per_px).sum())


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


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate(which: int, target_s: float, max_stamps: int, threads: int = 0, first: int = 0):
    """The FP64 oracle over a bounded sample of workload `which` (stamps
    first, first+1, ...), sized from a pilot run to about target_s seconds."""
    import oracle as O
    from paper_1203_0571_gb300 import synth
    O.build()
    # the thread count is set on every call: OpenMP keeps the last one set
    threads = threads if threads > 0 else (os.cpu_count() or 1)
    pilot = 64 if threads == 1 else 256
    sub = synth.make_workload(which, count=pilot, first=first)
    t = time.perf_counter()
    O.batch(sub.pix.numpy(), sub.offset.numpy(), sub.h.numpy(), sub.w.numpy(), threads=threads)
    dt = max(time.perf_counter() - t, 1e-3)
    count = int(min(max_stamps, max(pilot, pilot * target_s / dt)))
    sub = synth.make_workload(which, count=count, first=first)
    t = time.perf_counter()
    res, used = O.batch(sub.pix.numpy(), sub.offset.numpy(), sub.h.numpy(), sub.w.numpy(), threads=threads)
    dt = time.perf_counter() - t
    return count, dt, used, res


def cpu_oracle_rate(target_s: float, max_stamps: int):
    """The FP64 oracle on the host cores over a bounded sample of the workload,
    on all cores and on one (the paper timed one core of a 2.2 GHz CPU)."""
    count, dt, used, res = oracle_rate(WORKLOAD, target_s, max_stamps)
    c1, dt1, _, _ = oracle_rate(WORKLOAD, target_s / 3, max_stamps, threads=1)
    return {"value": count / dt, "unit": UNIT, "cores": used, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"first {count} stamps of the 100,000-stamp uniform-48px workload, "
                      f"whole chain, FP64, {used} threads, {dt:.2f} s wall",
            "single_core": {"value": c1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"first {c1} stamps, 1 thread, {dt1:.2f} s wall"},
            "it_mom_mean": float(np.mean(res["it_mom"])), "it_fit_mean": float(np.mean(res["it_fit"]))}


def run_oracle_rates(args):
    """Per-stamp oracle rates on seeded 10,000-stamp samples of the ragged,
    gradient and precision workloads (and the benchmark's), and on the whole
    256-stamp small workload, on all host cores and on one, bounded in time
    per sample; one JSON line."""
    from paper_1203_0571_gb300 import synth
    out = {"cpu": cpu_model(), "cores": os.cpu_count(), "kind": "oracle", "rates": {}}
    for which in (0, 1, 2, 3, 4, 5):
        name = synth.WORKLOADS[which].name
        cap = 10_000 if which else 256          # the small 32x32 workload whole
        n, dt, used, res = oracle_rate(which, 3 * args.cpu_seconds, cap)
        n1, dt1, _, _ = oracle_rate(which, args.cpu_seconds / 4, cap, threads=1)
        conv = ((res["status"] & 3) == 3).mean()
        out["rates"][name] = {"stamps": n, "threads": used, "stamps_per_s": n / dt, "s_per_stamp_1core": dt1 / n1,
                              "stamps_1core": n1, "converged_frac": float(conv),
                              "mean_px": float(res["npix"].mean())}
        print(json.dumps({name: out["rates"][name]}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)


def ragged_rate(ctx, B, synth, local, calls: int = 3):
    """The ragged workload (1,000,000 stamps, sides clip(round(8 r_e), 16, 128))
    through fse_fit_batch_ragged: size-class launches with autotuned shapes,
    captured once into a CUDA graph and replayed; CUDA events on the stream."""
    dev = f"cuda:{local}"
    rb = synth.make_workload(2, device=dev)
    ridx = B.make_index(rb.offset, rb.h, rb.w, device=dev)
    rout = torch.empty((rb.count, 64), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ctx.autotune(rb.pix, ridx, out=rout)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t
    gopts = B.default_opts(flags=B.FSE_FLAG_GRAPH)
    stream = torch.cuda.current_stream()
    ctx.fit_batch_ragged(rb.pix, ridx, out=rout, opts=gopts, stream=stream)   # captures the graph
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(calls):
        ctx.fit_batch_ragged(rb.pix, ridx, out=rout, opts=gopts, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / calls
    r = B.results(rout)
    px = int(rb.pix.numel())
    out = {"workload": "ragged-16-128px: 1,000,000 stamps, square side clip(round(8 r_e), 16, 128), "
                       "r_e logU[1,15] px, other parameters as the 32x32 workload, fp32, seed 2",
           "stamps": rb.count, "pixels": px, "value": rb.count / (ms / 1e3), "unit": "stamps/s",
           "px_per_s": px / (ms / 1e3), "ms_per_call": ms, "calls": calls,
           "launch": "seven size classes, three launches each, replayed as one CUDA graph, autotuned shapes",
           "autotune_s": tune_s, "converged_frac": float(((r["status"] & 3) == 3).mean())}
    del rb, ridx, rout
    torch.cuda.empty_cache()
    return out


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
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--oracle-rates", action="store_true",
                    help="time the oracle on samples of the other workloads (host cores only) and exit")
    args = ap.parse_args()
    if args.oracle_rates:
        return run_oracle_rates(args)
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
    sops = nominal_ops(res)
    kernel_ms = statistics.mean(step_ms)
    peak_gops = SMS * LANES_PER_SM * 2070.0 * 1e6 / 1e9     # at the maximum SM clock
    # achieved: the nominal per-pass figure x the pixel passes the launches ran
    # (the per-unit figure of the roofline contract); the builder's count of
    # the operations the kernels perform over the pixels they visit is beside it
    achieved = sops / (kernel_ms / 1e3) / 1e9
    achieved_builder = ops / (kernel_ms / 1e3) / 1e9
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

    ragged = None if args.no_ragged else ragged_rate(ctx, B, synth, local)

    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_oracle_rate(args.cpu_seconds, 40000)
    conv = (res["status"] & 3) == 3
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(n, world),
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": kernel_traffic(),
                     "frac_survey": achieved / peak_gops,
                     "ops_per_call_survey": sops,
                     "frac_builder": achieved_builder / peak_gops,
                     "ops_per_launch_builder": ops,
                     "accounting": "achieved: every pixel pass the three launches ran (start-up, moment "
                                   "passes and refinements, fit start, fit passes and refinements) at 31 "
                                   "(moment kind) or 33 (fit kind) operations per pixel of the whole stamp; "
                                   "frac_builder: the operations the kernels perform per pixel they visit, "
                                   "the moment passes over the weight's box",
                     "kernel": "estimator_kernel<startup> + <moments> + <fit> (the three launches of "
                               "one fse_fit_batch, f32)", "kernel_ms": kernel_ms,
                     "passes_per_stamp": {k: float(v.mean()) for k, v in pass_counts(res).items()},
                     "moment_box_frac": float((np.minimum(box_pixels(res, 48, 48), res["npix"]) /
                                               np.maximum(res["npix"], 1)).mean()),
                     "peak_source": "152 SMs x 128 fp32 lanes x 2070 MHz (issue slots, FMA = 1 op)"},
        "ragged": ragged,
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
