"""CUDA path against the FP64 oracle, through the C ABI (needs a GB300).

Parity gate: centroid 1e-4 px, e1/e2 1e-5, r_e/n/flux 1e-4 relative, chi^2
1e-5 relative, over every stamp that enters the gate (see tests/parity.py).
"""
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
def O(oracle):
    return oracle.get()


def opts_for(batch, **kw):
    """Options with the shared-memory tile sized to the batch's largest stamp."""
    return B.default_opts(max_pix=int((batch.h.to(torch.int64) * batch.w.to(torch.int64)).max()), **kw)


def gpu_run(ctx, batch, fn="fit_batch", inout=None, **kw):
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    kw.setdefault("opts", opts_for(batch))
    if inout is not None:
        out = torch.as_tensor(inout.view(np.uint8).reshape(-1, 64)).to("cuda")
        getattr(ctx, fn)(b.pix, idx, out, scale=b.scale, **kw)
    else:
        out = getattr(ctx, fn)(b.pix, idx, scale=b.scale, **kw)
    torch.cuda.synchronize()
    return B.results(out)


def assert_gate(rep, max_gpu_short_frac=0.01, max_subpixel_frac=0.01):
    """The parity gate of tests/parity.py: every gated stamp within tolerance,
    every exclusion and status disagreement confirmed by the oracle, at most
    max_gpu_short_frac of the stamps (rounded up) that the oracle converged
    and the GPU did not, and at most max_subpixel_frac of them disagreeing at
    the sub-pixel weight clamp, each listed with its reason."""
    PR.assert_gate(rep, max_gpu_short=int(np.ceil(max_gpu_short_frac * rep["n"])),
                   max_subpixel=int(np.ceil(max_subpixel_frac * rep["n"])))


def test_bn_table(ctx, O):
    n = torch.cat([torch.linspace(0.2, 10.0, 2001, dtype=torch.float64),
                   0.2 + 9.8 * torch.rand(2000, dtype=torch.float64, generator=torch.Generator().manual_seed(1))])
    b, db = ctx.sersic_b(n.cuda())
    b, db = b.cpu().numpy(), db.cpu().numpy()
    nn = n.numpy()
    rb = np.array([O.sersic_b(x) for x in nn])
    rdb = np.array([O.sersic_db(x) for x in nn])
    # the fit uses b in fp32 (resolution 6e-8); the table is held 100x finer than that
    assert np.max(np.abs(b / rb - 1)) <= 5e-10
    assert np.max(np.abs(db / rdb - 1)) <= 1e-6


def test_small_workload_chain(ctx, O):
    batch = synth.make_workload(0)
    g = gpu_run(ctx, batch)
    ids = np.arange(batch.count)
    o = PR.oracle_results(O, batch, ids)
    rep = PR.compare(g, o, O=O, batch=batch, ids=ids)
    PR.dump("small_chain", rep)
    assert_gate(rep)


def test_stage_centroid(ctx, O):
    batch = synth.make_workload(0)
    g = gpu_run(ctx, batch, "centroid")
    o = PR.oracle_results(O, batch, np.arange(batch.count), stage="centroid")
    rep = PR.compare(g, o, keys=("x0", "y0"), fit=False, O=O, batch=batch, ids=np.arange(batch.count),
                     ellip=False)
    PR.dump("stage_centroid", rep)
    assert_gate(rep)
    both = ((g["status"] & 1) & (o["status"] & 1)).astype(bool)
    assert np.max(np.abs(g["r50"][both] / o["r50"][both] - 1)) <= 1e-6
    assert np.max(np.abs(g["sigma_w"][both] / o["sigma_w"][both] - 1)) <= 1e-6


def test_stage_ellipticity(ctx, O):
    batch = synth.make_workload(0)
    ids = np.arange(batch.count)
    gc = gpu_run(ctx, batch, "centroid")
    ge = gpu_run(ctx, batch, "ellipticity", inout=gc.copy())
    oc = PR.oracle_results(O, batch, ids, stage="centroid")
    oe = PR.oracle_results(O, batch, ids, stage="ellipticity", init=oc)
    rep = PR.compare(ge, oe, keys=("x0", "y0", "e1", "e2"), fit=False, O=O, batch=batch, ids=ids)
    PR.dump("stage_ellipticity", rep)
    assert_gate(rep)


def test_stage_fit_isolated(ctx, O):
    """The fit alone, both sides started from the oracle's centre and ellipticity."""
    batch = synth.make_workload(0)
    ids = np.arange(batch.count)
    om = PR.oracle_results(O, batch, ids)
    inout = np.zeros(batch.count, dtype=B.RESULT_DTYPE)
    for k in ("x0", "y0", "e1", "e2", "sigma_w"):
        inout[k] = om[k].astype(np.float32)
    inout["status"] = om["status"] & 1
    g = gpu_run(ctx, batch, "sersic_fit", inout=inout)
    init = np.zeros(batch.count, dtype=om.dtype)
    for k in ("x0", "y0", "e1", "e2", "sigma_w"):
        init[k] = inout[k].astype(np.float64)      # the same fp32-rounded start
    init["status"] = inout["status"]
    o = PR.oracle_results(O, batch, ids, stage="fit", init=init)
    rep = PR.compare(g, o, keys=("re", "n", "flux", "chi2"), O=O, batch=batch, ids=ids)
    PR.dump("stage_fit", rep)
    assert_gate(rep)


def test_uniform_workload_full_size_sampled(ctx, O):
    """100,000 stamps of 48x48 in the benchmark's launch; 400 sampled stamps checked."""
    batch = synth.make_workload(1, device="cuda")
    idx = B.make_index(batch.offset, batch.h, batch.w)
    out = ctx.fit_batch(batch.pix, idx, opts=B.default_opts(max_pix=48 * 48))
    torch.cuda.synchronize()
    g = B.results(out)
    assert (g["npix"] == 48 * 48).all()
    assert not (g["status"] & (B.ST["BAD_SIZE"] | B.ST["NONFINITE"] | B.ST["TIMEOUT"])).any()
    conv = (g["status"] & 3) == 3
    assert conv.mean() > 0.9
    for k in ("x0", "y0", "e1", "e2", "I0", "re", "n", "flux", "chi2"):
        assert np.isfinite(g[k][conv]).all(), k
    ids = np.sort(np.random.default_rng(7).choice(batch.count, 400, replace=False))
    cpu = synth.make_workload(1, ids=ids)
    o = PR.oracle_results(O, cpu, np.arange(ids.size))
    rep = PR.compare(g[ids], o, O=O, batch=cpu, ids=np.arange(ids.size))
    PR.dump("uniform_sampled", rep)
    assert_gate(rep)


def test_ragged_unaligned(ctx, O):
    batch = synth.make_workload(2, count=3000)
    assert (batch.offset.numpy() % 4 != 0).mean() > 0.5      # most stamps start unaligned
    g = gpu_run(ctx, batch)
    ids = np.sort(np.random.default_rng(3).choice(batch.count, 300, replace=False))
    o = PR.oracle_results(O, batch, ids)
    rep = PR.compare(g[ids], o, O=O, batch=batch, ids=ids)
    PR.dump("ragged", rep)
    assert_gate(rep)


def test_bf16_pixels(ctx, O):
    batch = synth.encode_bf16(synth.make_workload(4, count=400))
    g = gpu_run(ctx, batch)
    ids = np.arange(batch.count)
    o = PR.oracle_results(O, batch, ids)
    rep = PR.compare(g, o, O=O, batch=batch, ids=ids)
    PR.dump("bf16", rep)
    assert_gate(rep)


def test_inverse_variance(ctx, O):
    batch = synth.make_workload(0)
    ivar = (0.5 + 1.5 * torch.rand(batch.pix.numel(), generator=torch.Generator().manual_seed(4))).float()
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    g = B.results(ctx.fit_batch(b.pix, idx, inv_var=ivar.cuda(), opts=opts_for(batch)))
    ids = np.arange(batch.count)
    iv = ivar.numpy()
    o = PR.oracle_results(O, batch, ids, ivar=iv)
    rep = PR.compare(g, o, O=O, batch=batch, ids=ids, ivar=iv)
    PR.dump("inv_var", rep)
    assert_gate(rep)


def test_edge_cases(ctx, O):
    rng = np.random.default_rng(0)
    good = synth.single_stamp(32, 32, n=1.5, re=3.0, g1=0.2, g2=0.1, xc=15.3, yc=16.1, I0=500.0,
                              noise_sigma=1.0, seed=1)
    big = synth.single_stamp(128, 128, n=2.0, re=9.0, g1=-0.1, g2=0.3, xc=63.6, yc=64.2, I0=200.0,
                             noise_sigma=1.0, seed=2)
    nan = good.copy()
    nan[5, 7] = np.nan
    stamps = [good, nan, np.zeros((32, 32)), rng.normal(size=(1, 1)) + 5, rng.normal(size=(3, 5)) + 3,
              np.ones((129, 129)), big, rng.normal(size=(17, 23)) + 1]
    pix = np.concatenate([s.astype(np.float32).ravel() for s in stamps])
    offs = np.cumsum([0] + [s.size for s in stamps[:-1]])
    hs = np.array([s.shape[0] for s in stamps])
    ws = np.array([s.shape[1] for s in stamps])
    idx = B.make_index(offs, hs, ws)
    g = B.results(ctx.fit_batch(torch.as_tensor(pix).cuda(), idx))
    o, _ = O.batch(pix, offs, hs, ws)
    assert g["status"][1] & B.ST["NONFINITE"] and o["status"][1] & 16
    assert g["status"][2] & B.ST["INIT_FALLBACK"] and g["status"][2] & B.ST["MOM_FAILED"]
    assert g["status"][5] == B.ST["BAD_SIZE"] and o["status"][5] == 32
    for j in (0, 6):
        rep = PR.compare(g[j:j + 1], o[j:j + 1])
        assert rep["gated"] == 1 and rep["within_tolerance"] == 1, (j, rep["max_err"])
    # moment-only agreement of the tiny stamps where both converge
    for j in (3, 4, 7):
        if (g["status"][j] & 1) and (o["status"][j] & 1):
            assert abs(g["x0"][j] - o["x0"][j]) <= 1e-4 and abs(g["y0"][j] - o["y0"][j]) <= 1e-4
    # an empty batch is a no-op
    empty = ctx.fit_batch(torch.zeros(1, device="cuda"), B.make_index([], [], []))
    assert empty.shape[0] == 0


def test_plain_equals_batched(ctx):
    batch = synth.make_workload(1, count=1000)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    o1 = ctx.fit_batch(b.pix, idx, opts=opts_for(batch))
    o2 = ctx.fit_batch_plain(b.pix, idx, opts=opts_for(batch))
    o3 = ctx.fit_batch(b.pix, idx, opts=opts_for(batch, warps_per_cta=1))
    # the full 128x128 tile, still one warp per stamp (several warps sum in
    # another order: tests/test_gpu_multiwarp.py)
    o4 = ctx.fit_batch(b.pix, idx, opts=B.default_opts(warps_per_stamp=1))
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(o1, o3) and torch.equal(o1, o4)


def test_host_buffers_equal_device(ctx):
    batch = synth.make_workload(1, count=10000)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    dev = B.results(ctx.fit_batch(b.pix, idx, opts=opts_for(batch)))
    host_pix = batch.pix.pin_memory()
    host_idx = B.make_index(batch.offset, batch.h, batch.w, device="cpu").pin_memory()
    out = torch.zeros((batch.count, 64), dtype=torch.uint8).pin_memory()
    ctx.fit_batch_host(host_pix, host_idx, out=out)
    host = out.numpy().view(B.RESULT_DTYPE).reshape(-1)
    assert host.tobytes() == dev.tobytes()


def test_host_buffers_stamp_outside_the_buffer(ctx):
    """A stamp past the end of the pixel buffer in the last of the nine chunks:
    the call returns FSE_EINVAL with out[] untouched, after the chunks before
    it were checked and copied; the context then runs the batch unchanged."""
    batch = synth.make_workload(1, count=9000)
    host_pix = batch.pix.pin_memory()
    bad = B.make_index(batch.offset, batch.h, batch.w, device="cpu").clone()
    bad[8990, 0] = batch.pix.numel() - 100          # offset + 48 * 48 > npix_total
    out = torch.full((batch.count, 64), 0xA5, dtype=torch.uint8).pin_memory()
    with pytest.raises(B.FseError) as err:
        ctx.fit_batch_host(host_pix, bad.pin_memory(), out=out)
    assert err.value.code == B.FSE_EINVAL and "8990" in str(err.value)
    assert bool((out == 0xA5).all())
    good = B.make_index(batch.offset, batch.h, batch.w, device="cpu").pin_memory()
    ctx.fit_batch_host(host_pix, good, out=out)
    b = batch.to("cuda")
    dev = B.results(ctx.fit_batch(b.pix, B.make_index(b.offset, b.h, b.w), opts=opts_for(batch)))
    assert out.numpy().view(B.RESULT_DTYPE).reshape(-1).tobytes() == dev.tobytes()


def test_host_buffers_ragged_bf16_inverse_variance(ctx):
    """The chunked host-buffer pipeline on 9,001 stamps of 32-64 px (bf16 with a
    per-stamp scale, a per-pixel inverse variance, two stamps of a refused
    size): its results equal fse_fit_batch on device buffers, byte for byte."""
    batch = synth.encode_bf16(synth.make_workload(4, count=9001))
    opts = opts_for(batch)
    batch.h[17] = 0                     # empty: BAD_SIZE
    batch.h[5000], batch.w[5000] = 1, 129   # a side above the limit: BAD_SIZE
    rng = np.random.default_rng(11)
    ivar = torch.as_tensor(rng.uniform(0.5, 2.0, batch.pix.numel()).astype(np.float32))
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    dev = B.results(ctx.fit_batch(b.pix, idx, scale=b.scale, inv_var=ivar.cuda(), opts=opts))
    host_idx = B.make_index(batch.offset, batch.h, batch.w, device="cpu").pin_memory()
    out = torch.zeros((batch.count, 64), dtype=torch.uint8).pin_memory()
    ctx.fit_batch_host(batch.pix.pin_memory(), host_idx, scale=batch.scale.pin_memory(),
                       inv_var=ivar.pin_memory(), opts=opts, out=out)
    host = out.numpy().view(B.RESULT_DTYPE).reshape(-1)
    assert host["status"][17] & B.ST["BAD_SIZE"] and host["status"][5000] & B.ST["BAD_SIZE"]
    assert host.tobytes() == dev.tobytes()


def test_fixed_gain_reaches_the_same_fixed_point(ctx, O):
    """k = 0.75 (the fixed gain of Sec. 2) and the default determined gain both
    reach the oracle's fixed point; only the number of passes differs."""
    batch = synth.make_workload(0)
    ids = np.arange(batch.count)
    o = PR.oracle_results(O, batch, ids)
    g75 = gpu_run(ctx, batch, opts=opts_for(batch, k_gain=0.75))
    g0 = gpu_run(ctx, batch)
    for name, g in (("k075", g75), ("k_newton", g0)):
        rep = PR.compare(g, o, O=O, batch=batch, ids=ids)
        PR.dump(f"gain_{name}", rep)
        assert_gate(rep)
    both = ((g75["status"] & 1) & (g0["status"] & 1)).astype(bool)
    assert g0["it_mom"][both].mean() < g75["it_mom"][both].mean()


def test_side_limit(ctx, O):
    """Stamps with a side above 128 pixels are refused (BAD_SIZE) whatever their
    area, by the estimator and by the oracle's batch; stamps of the same batch
    within the limit, including elongated ones, are measured as usual."""
    rng = np.random.default_rng(12)
    shapes = [(1, 200), (200, 1), (2, 1200), (129, 100), (24, 96), (48, 48), (128, 40), (40, 128)]
    stamps = []
    for h, w in shapes:
        yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
        xc, yc = rng.uniform(0.4, 0.6) * (w - 1), rng.uniform(0.4, 0.6) * (h - 1)
        stamps.append(50.0 * np.exp(-((xx - xc) ** 2 + (yy - yc) ** 2) / (2 * 3.0 ** 2)) +
                      rng.normal(0, 0.2, (h, w)))
    pix = np.concatenate([s_.astype(np.float32).ravel() for s_ in stamps])
    offs = np.cumsum([0] + [s_.size for s_ in stamps[:-1]])
    hs = np.array([s_.shape[0] for s_ in stamps])
    ws = np.array([s_.shape[1] for s_ in stamps])
    idx = B.make_index(offs, hs, ws)
    d = torch.as_tensor(pix).cuda()
    g = B.results(ctx.centroid(d, idx, opts=B.default_opts(max_pix=16384)))
    gf = B.results(ctx.fit_batch(d, idx, opts=B.default_opts(max_pix=16384)))
    o, _ = O.batch(pix, offs, hs, ws, stage="centroid")
    for j, (h, w) in enumerate(shapes):
        if h > 128 or w > 128:
            assert g["status"][j] == gf["status"][j] == B.ST["BAD_SIZE"] and o["status"][j] == 32, (h, w)
            continue
        assert abs(g["r50"][j] / o["r50"][j] - 1) <= 1e-6, (h, w, g["r50"][j], o["r50"][j])
        assert (g["status"][j] & 1) and (o["status"][j] & 1), (h, w)
        assert abs(g["x0"][j] - o["x0"][j]) <= 1e-4 and abs(g["y0"][j] - o["y0"][j]) <= 1e-4, (h, w)


@pytest.mark.parametrize("case", ["small-32px", "uniform-48px"])
def test_matched_weight_chain(ctx, O, case):
    """The whole chain with the matched-weight rule sigma_w^2 = sum I W R^2 /
    sum I W (the weight-size iteration of Sec. 4.2.1 applied to the weight of
    Secs. 2-3; fse_opts.sigw_mode = 0) on both sides: 256 stamps of 32x32 and
    400 stamps sampled from the 48x48 workload."""
    if case == "small-32px":
        batch = synth.make_workload(0)
    else:
        ids = np.sort(np.random.default_rng(21).choice(100_000, 400, replace=False))
        batch = synth.make_workload(1, ids=ids)
    g = gpu_run(ctx, batch, opts=opts_for(batch, sigw_mode=0))
    ids = np.arange(batch.count)
    oo = O.default_opts(sigw_mode=0)
    o = PR.oracle_results(O, batch, ids, opts=oo)
    rep = PR.compare(g, o, O=O, batch=batch, ids=ids, sigw_mode=0, orc_opts=oo)
    PR.dump(f"matched_{case}", rep)
    # cuspy galaxies drive the matched weight to its 0.5 px clamp, below the
    # pixel scale, where the iteration has several fixed points: measured 12 of
    # 256 and 15 of 400 stamps whose convergence differs there
    assert_gate(rep, max_subpixel_frac=0.08)
    # the weight size is the matched one on both sides, where it is not clamped
    # (57 % of the small workload's stamps; the cuspier rest reach the 0.5 px clamp)
    both = (((g["status"] & 1) & (o["status"] & 1)) != 0) & ((g["status"] & B.ST["SIGW_CLAMPED"]) == 0)
    assert both.mean() > 0.5
    assert np.max(np.abs(g["sigma_w"][both] / o["sigma_w"][both] - 1)) <= 1e-5


def test_growth_curve_far_from_the_brightest_pixel(ctx, O):
    """The start-up's growth curve (Sec. 4.1) when the brightest pixel is far
    from the stamp's centre, in every quadrant: a bright spike on a broad
    galaxy, so that half the light is enclosed only at rings reaching towards
    the far corners.  r50 and the start (the brightest pixel) agree with the
    oracle whichever corner the spike is nearest."""
    rng = np.random.default_rng(31)
    spikes = [(40, 40), (5, 44), (44, 3), (46, 46), (1, 1), (24, 46), (46, 24), (3, 3), (30, 2)]
    stamps = []
    for (sy, sx) in spikes:
        img = synth.single_stamp(48, 48, n=1.0, re=9.0, g1=0.1, g2=-0.05, xc=23.6, yc=24.3, I0=40.0,
                                 noise_sigma=1.0, seed=int(rng.integers(1 << 30)))
        img[sy, sx] += 500.0
        stamps.append(img)
    pix = np.concatenate([s_.astype(np.float32).ravel() for s_ in stamps])
    n = len(stamps)
    offs = np.arange(n) * 48 * 48
    idx = B.make_index(offs, [48] * n, [48] * n)
    g = B.results(ctx.centroid(torch.as_tensor(pix).cuda(), idx, opts=B.default_opts(max_pix=48 * 48)))
    o, _ = O.batch(pix, offs, np.full(n, 48), np.full(n, 48), stage="centroid")
    for j, (sy, sx) in enumerate(spikes):
        assert np.isfinite(o["r50"][j]) and o["r50"][j] > 5.0, (sy, sx, o["r50"][j])
        assert abs(g["r50"][j] / o["r50"][j] - 1) <= 1e-6, (sy, sx, g["r50"][j], o["r50"][j])
        start_bits = B.ST["NONFINITE"] | B.ST["BAD_SIZE"] | B.ST["INIT_FALLBACK"] | B.ST["SIGW_CLAMPED"]
        assert (int(g["status"][j]) ^ int(o["status"][j])) & start_bits == 0, (sy, sx, g["status"][j], o["status"][j])
        assert (g["x0"][j], g["y0"][j]) == (sx, sy) or g["status"][j] & 1
