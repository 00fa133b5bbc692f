"""The chi^2 adjoint (fse_sersic_chi2_grad) against the FP64 oracle's gradient,
through the C ABI and the autograd bridge (needs a GB300).

Tolerance, derived from the arithmetic: the kernel evaluates each pixel's
model m and residual r in fp32 (MUFU exp2/log2 plus about 20 dependent
operations), so m and r carry relative errors of a few 1e-7; the exponent
b u (up to about 20 at the stamp edge for n = 6) multiplies the error of u,
and the per-lane fp32 sums of about 128 terms add about 1e-6 of the absolute
sum.  The oracle returns, per output, the first-order scale
S = sum 2 w |dm/dp| (|m| + |r|) (and sum 2 w |r| (|m| + |r|) for chi^2); an
evaluation with per-pixel relative error eps differs by at most about
eps * S.  The test takes eps = 4e-6 for chi^2 and d chi^2/dp.

Per pixel, the model's exponent b u = ln(I0 / m) multiplies the relative error
of u (MUFU exp2 and log2, a few 1e-7), so m carries a relative error of about
4e-7 (1 + ln(I0/|m|)); the pixel gradient -2 w r is checked against
2 w |m| 1e-6 (1 + ln(I0/|m|)) + 1e-6 |d chi^2/dI|.
"""
import numpy as np
import pytest
import torch

from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth
from paper_1203_0571_gb300.autograd import sersic_chi2

pytestmark = pytest.mark.gpu
EPS = 4e-6


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return B.Context(0)


@pytest.fixture(scope="module")
def O(oracle):
    return oracle.get()


def true_params(batch, perturb=True):
    t = batch.truth
    p = np.stack([t["xc"], t["yc"], t["g1"], t["g2"], t["I0"], t["re"], t["n"]], axis=1)
    if perturb:
        # every other stamp away from its generating point, so residuals are not pure noise
        k = np.arange(batch.count) % 2 == 1
        p[k] *= np.array([1.0, 1.0, 1.0, 1.0, 0.97, 1.04, 0.95])
        p[k, 0] += 0.06
        p[k, 1] -= 0.04
        p[k, 2] += 0.015
    return p.astype(np.float32)


def gpu_grad(ctx, batch, p32, ivar=None, dpix=True):
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    chi2, dpar, dp = ctx.chi2_grad(b.pix, idx, torch.as_tensor(p32).cuda(), scale=b.scale,
                                   inv_var=None if ivar is None else torch.as_tensor(ivar).cuda(),
                                   want_dpix=dpix)
    torch.cuda.synchronize()
    return (chi2.cpu().numpy(), dpar.cpu().numpy(), None if dp is None else dp.cpu().numpy())


def check_against_oracle(O, batch, p32, chi2, dpar, dpix, ivar=None):
    worst = 0.0
    for s in range(batch.count):
        img = batch.stamp(s)
        o = int(batch.offset[s])
        hh, ww = img.shape
        iv = None if ivar is None else ivar[o:o + hh * ww].reshape(hh, ww).astype(np.float64)
        c, g, dp, sc = O.chi2_grad(img, p32[s].astype(np.float64), ivar=iv, pixels=True, scales=True)
        assert abs(chi2[s] - c) <= EPS * sc[7], (s, chi2[s], c, sc[7])
        err = np.abs(dpar[s] - g)
        assert np.all(err <= EPS * sc[:7]), (s, dpar[s], g, sc[:7])
        worst = max(worst, float(np.max(err / np.maximum(sc[:7], 1e-300))))
        if dpix is not None:
            gp = dpix[o:o + hh * ww].reshape(hh, ww)
            w_ = 1.0 if iv is None else iv
            m = np.abs(img - dp / (2.0 * w_))                 # |model| from r = -dp / 2w
            bu = np.log(np.maximum(abs(float(p32[s][4])) / np.maximum(m, 1e-300), 1.0))
            tol = 2.0 * w_ * m * 1e-6 * (1.0 + bu) + 1e-6 * np.abs(dp) + 1e-30
            bad = np.abs(gp - dp) > tol
            if bad.any():
                k = np.unravel_index(np.argmax(np.abs(gp - dp) / tol), gp.shape)
                raise AssertionError(("pixel", s, k, float(gp[k]), float(dp[k]), float(img[k]),
                                      float(tol[k]), int(bad.sum()), p32[s].tolist()))
    return worst


def test_adjoint_matches_oracle_grad64(ctx, O):
    """65,536-stamp workload's first 96 stamps (64x64, n up to 6), half at the
    generating parameters, half away from them."""
    batch = synth.make_workload(3, count=96)
    p32 = true_params(batch)
    chi2, dpar, dpix = gpu_grad(ctx, batch, p32)
    worst = check_against_oracle(O, batch, p32, chi2, dpar, dpix)
    print("worst |gpu - oracle| / scale:", worst)


def test_adjoint_inverse_variance_and_bf16(ctx, O):
    batch = synth.make_workload(3, count=24)
    p32 = true_params(batch)
    ivar = (0.5 + np.random.default_rng(8).random(batch.pix.numel())).astype(np.float32)
    chi2, dpar, dpix = gpu_grad(ctx, batch, p32, ivar=ivar)
    check_against_oracle(O, batch, p32, chi2, dpar, dpix, ivar=ivar)
    bb = synth.encode_bf16(batch)
    chi2, dpar, dpix = gpu_grad(ctx, bb, p32)
    check_against_oracle(O, bb, p32, chi2, dpar, dpix)


def test_adjoint_against_finite_differences(ctx, O):
    """Central differences of the FP64 chi^2 with h = 1e-3 of each parameter's
    scale (1 px for the centre, 0.1 for e, |p| otherwise), Richardson-combined
    with h/2, against the GPU gradient."""
    batch = synth.make_workload(3, count=6)
    p32 = true_params(batch)
    _, dpar, _ = gpu_grad(ctx, batch, p32, dpix=False)
    for s in range(batch.count):
        img = batch.stamp(s)
        p = p32[s].astype(np.float64)
        _, g, sc = O.chi2_grad(img, p, scales=True)
        step = 1e-3 * np.array([1.0, 1.0, 0.1, 0.1, abs(p[4]), p[5], p[6]])
        for a in range(7):
            if a in (2, 3) and np.hypot(p[2], p[3]) < 0.01:
                continue            # the |g| kink
            def f(h):
                q = p.copy()
                q[a] += h
                return O.chi2_grad(img, q)[0]
            d1 = (f(step[a]) - f(-step[a])) / (2 * step[a])
            d2 = (f(step[a] / 2) - f(-step[a] / 2)) / step[a]
            fd = (4 * d2 - d1) / 3
            assert abs(dpar[s, a] - fd) <= EPS * sc[a] + 1e-6 * abs(fd), (s, a, dpar[s, a], fd)


def test_vjp_and_autograd(ctx):
    batch = synth.make_workload(3, count=64)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    p = torch.as_tensor(true_params(batch)).cuda()
    chi2, dpar, dpix = ctx.chi2_grad(b.pix, idx, p, want_dpix=True)
    gout = torch.linspace(-2.0, 3.0, batch.count, dtype=torch.float64, device="cuda")
    _, vpar, vpix = ctx.chi2_grad(b.pix, idx, p, gout=gout, want_chi2=False, want_dpix=True)
    # the kernel applies gout[s] (rounded to fp32) as the last multiply
    assert torch.equal(vpar, dpar * gout.float()[:, None])
    rows = torch.repeat_interleave(gout.float(), (b.h * b.w).long())
    assert torch.equal(vpix, dpix * rows)
    # autograd: forward equals chi2, backward equals the VJP
    pp = p.clone().requires_grad_(True)
    px = b.pix.clone().requires_grad_(True)
    out = sersic_chi2(pp, px, idx, ctx)
    # the chi^2-only instance of the kernel gives the same chi^2 bit for bit
    assert torch.equal(out.detach(), chi2)
    (out * gout).sum().backward()
    assert torch.equal(pp.grad, vpar) and torch.equal(px.grad, vpix)


def test_invalid_parameters_and_empty(ctx):
    batch = synth.make_workload(3, count=4)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    p = torch.as_tensor(true_params(batch, perturb=False)).cuda()
    p[0, 5] = -1.0          # r_e <= 0
    p[1, 2] = 0.9
    p[1, 3] = 0.9           # |g| >= 1
    p[2, 6] = 20.0          # n outside the b(n) table
    chi2, dpar, dpix = ctx.chi2_grad(b.pix, idx, p, want_dpix=True)
    assert torch.isnan(chi2[:3]).all() and torch.isnan(dpar[:3]).all()
    assert torch.isfinite(chi2[3]) and torch.isfinite(dpar[3]).all()
    n0 = int(b.h[0] * b.w[0])
    assert torch.isnan(dpix[:3 * n0]).all() and torch.isfinite(dpix[3 * n0:]).all()
    e = ctx.chi2_grad(b.pix, B.make_index([], [], []), torch.zeros((0, 7), device="cuda"))
    assert e[0].numel() == 0


def test_adjoint_round_and_axis_aligned(ctx, O):
    """g = 0 (the kink: d|g|/dg taken as 0 on both sides) and ellipses whose
    major axis lies along x (phi = 0), y (phi = 90 deg) or a diagonal."""
    gs = [(0.0, 0.0), (0.3, 0.0), (-0.3, 0.0), (0.0, 0.3), (0.0, -0.3), (0.2, 0.2)]
    stamps, params = [], []
    for k, (g1, g2) in enumerate(gs):
        img = synth.single_stamp(40, 36, n=1.7, re=3.2, g1=g1, g2=g2, xc=17.3, yc=19.6, I0=900.0,
                                 noise_sigma=1.0, seed=90 + k)
        stamps.append(img.astype(np.float32))
        params.append([17.35, 19.55, g1, g2, 880.0, 3.3, 1.6])
    pix = np.concatenate([s_.ravel() for s_ in stamps])
    offs = np.arange(len(stamps)) * 40 * 36
    idx = B.make_index(offs, [40] * len(stamps), [36] * len(stamps))
    p32 = np.asarray(params, dtype=np.float32)
    chi2, dpar, dpix = ctx.chi2_grad(torch.as_tensor(pix).cuda(), idx, torch.as_tensor(p32).cuda(),
                                     want_dpix=True)
    chi2, dpar = chi2.cpu().numpy(), dpar.cpu().numpy()
    for s_, img in enumerate(stamps):
        c, g, sc = O.chi2_grad(img.astype(np.float64), p32[s_].astype(np.float64), scales=True)
        assert abs(chi2[s_] - c) <= EPS * sc[7], (s_, chi2[s_], c)
        assert np.all(np.abs(dpar[s_] - g) <= EPS * sc[:7]), (s_, dpar[s_], g, sc[:7])
