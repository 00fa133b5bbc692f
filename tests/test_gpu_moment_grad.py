"""Implicit gradients of the moment fixed point (Secs. 2-3) on the GPU
(fse_moment_vjp / fse_moment_jvp) against the FP64 oracle, needs a GB300.

Both sides evaluate the derivatives at the same theta: the oracle's fixed point
rounded into the library's fp32 result records.  The kernel forms J from 15
weighted moments accumulated in fp32 (double-float per lane), so J carries a
relative error of a few 1e-7 of its norm; the Jacobi-scaled J of these stamps
has condition numbers 1-15, so lambda = J^-T v, and with it the pixel
gradient, is good to about 1e-6 of its largest entry.  Tolerance: 2e-5 of the
stamp's largest |dL/dI| per pixel (VJP) and of the largest |dtheta| per
component (JVP), times max(1, cond/10), times max(1, 1/(5 q)) with
q = (1 - |g|)/(1 + |g|) the axis ratio of the weight: the moments of a weight
elongated by 1/q cancel in the assembly of J by up to about 1/q.
"""
import numpy as np
import pytest
import torch

import parity as PR
from paper_1203_0571_gb300 import binding as B
from paper_1203_0571_gb300 import synth

pytestmark = pytest.mark.gpu

ST = B.ST
TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    return B.Context(0)


@pytest.fixture(scope="module")
def O(oracle):
    return oracle.get()


def oracle_fixed_point(O, batch, sigw_mode, ellip=True):
    """The oracle's moment stage (Sec. 2, then Sec. 3), as fp32 result records."""
    ids = np.arange(batch.count)
    o = O.default_opts(sigw_mode=sigw_mode)
    r = PR.oracle_results(O, batch, ids, "centroid", opts=o)
    if ellip:
        r = PR.oracle_results(O, batch, ids, "ellipticity", init=r, opts=o)
    out = np.zeros(len(r), dtype=B.RESULT_DTYPE)
    for k in B.RESULT_DTYPE.names:
        out[k] = r[k]
    if not ellip:
        out["e1"] = out["e2"] = 0.0
    return out


def theta32(rec):
    return np.array([float(np.float32(rec[k])) for k in ("x0", "y0", "e1", "e2", "sigma_w")])


def oracle_mode(O, mode, rec):
    """The oracle's mode bits for one stamp: a clamped sigma_w is held."""
    m = (O.MOM_ELLIP if mode & B.FSE_MOM_ELLIP else 0)
    if int(rec["status"]) & ST["SIGW_CLAMPED"] or mode & B.FSE_MOM_SIGW_FIXED:
        return m | O.MOM_SIGW_FIXED
    return m | (O.MOM_SIGW_R50 if mode & B.FSE_MOM_SIGW_R50 else 0)


def cond_scaled(O, I, th, om):
    _, J = O.moment_jacobian(I, th)
    act = [0, 1] + ([2, 3] if om & O.MOM_ELLIP else []) + \
        ([4] if not om & (O.MOM_SIGW_FIXED | O.MOM_SIGW_R50) else [])
    Ja = J[np.ix_(act, act)]
    d = np.sqrt(np.abs(np.diag(Ja)))
    if not np.all(d > 0):
        return np.inf
    sv = np.linalg.svd(Ja / np.outer(d, d), compute_uv=False)
    return float(sv[0] / sv[-1])


def run_case(ctx, O, batch, mode, sigw_mode, seed):
    ellip = bool(mode & B.FSE_MOM_ELLIP)
    rec = oracle_fixed_point(O, batch, sigw_mode, ellip)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(batch.count, 5)).astype(np.float32)
    tangent = rng.normal(size=batch.pix.numel()).astype(np.float32)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    moments = torch.as_tensor(rec.view(np.uint8).reshape(-1, 64)).to("cuda")
    st_v = torch.zeros(batch.count, dtype=torch.int32, device="cuda")
    st_j = torch.zeros(batch.count, dtype=torch.int32, device="cuda")
    dpix = ctx.moment_vjp(b.pix, idx, moments, torch.as_tensor(v).cuda(), mode=mode, scale=b.scale,
                          status=st_v).cpu().numpy()
    dth = ctx.moment_jvp(b.pix, idx, moments, torch.as_tensor(tangent).cuda(), mode=mode, scale=b.scale,
                         status=st_j).cpu().numpy()
    st_v, st_j = st_v.cpu().numpy(), st_j.cpu().numpy()
    assert np.array_equal(st_v, st_j)
    worst, checked = [0.0, 0.0], 0
    for i in range(batch.count):
        o, hh, ww = int(batch.offset[i]), int(batch.h[i]), int(batch.w[i])
        if not int(rec["status"][i]) & ST["MOM_CONVERGED"]:
            assert st_v[i] == ST["MOM_FAILED"] and not np.any(dpix[o:o + hh * ww]), i
            continue
        I = batch.stamp(i).astype(np.float32)
        th = theta32(rec[i])
        om = oracle_mode(O, mode, rec[i])
        vv = v[i].astype(np.float64)
        if not ellip:
            vv[2:4] = 0.0
        dI, sing = O.moment_vjp(I, th, vv, mode=om)
        u = tangent[o:o + hh * ww].reshape(hh, ww).astype(np.float64)
        d, sing2 = O.moment_jvp(I, th, u, mode=om)
        cond = cond_scaled(O, I, th, om)
        if sing or cond > 1e5:
            continue
        assert st_v[i] == 0, (i, st_v[i])
        ga = np.hypot(th[2], th[3])
        tol = TOL * max(1.0, cond / 10) * max(1.0, (1 + ga) / (5 * (1 - ga)))
        g = dpix[o:o + hh * ww].reshape(hh, ww)
        e = np.abs(g - dI).max() / np.abs(dI).max()
        ej = np.abs(dth[i] - d).max() / np.abs(d).max()
        worst = [max(worst[0], e / tol), max(worst[1], ej / tol)]
        assert e <= tol, (i, e, tol, cond)
        assert ej <= tol, (i, dth[i], d, tol, cond)
        checked += 1
    print("checked", checked, "of", batch.count, "worst error / tolerance (vjp, jvp)", worst, flush=True)
    assert checked >= 0.9 * batch.count
    return dpix, dth


@pytest.mark.parametrize("which,count", [(0, 256), (1, 400), (2, 300)])
@pytest.mark.parametrize("sigw_mode", [1, 0])
def test_moment_grad_matches_oracle(ctx, O, which, count, sigw_mode):
    """Secs. 2-3 fixed point; sigma_w from the growth curve (sigw_mode 1) or
    the matched weight (0); 32x32, 48x48 and ragged 16-128 px stamps."""
    mode = B.FSE_MOM_ELLIP | (B.FSE_MOM_SIGW_R50 if sigw_mode == 1 else 0)
    run_case(ctx, O, synth.make_workload(which, count=count), mode, sigw_mode, seed=which)


@pytest.mark.parametrize("sigw_mode", [1, 0])
def test_moment_grad_centroid_stage(ctx, O, sigw_mode):
    """Sec. 2 alone (g = 0 held): theta = (x0, y0, sigma_w)."""
    mode = B.FSE_MOM_SIGW_R50 if sigw_mode == 1 else 0
    run_case(ctx, O, synth.make_workload(1, count=300, first=1000), mode, sigw_mode, seed=7)


def test_moment_grad_bf16(ctx, O):
    batch = synth.encode_bf16(synth.make_workload(1, count=300, first=2000))
    run_case(ctx, O, batch, B.FSE_MOM_ELLIP | B.FSE_MOM_SIGW_R50, 1, seed=9)


def test_moment_grad_sigma_held(ctx, O):
    batch = synth.make_workload(0, count=128)
    run_case(ctx, O, batch, B.FSE_MOM_ELLIP | B.FSE_MOM_SIGW_FIXED, 0, seed=5)


def _gaussian_batch(count, h, w, seed):
    """Noiseless elliptical Gaussians exp(-R^2/2 s^2) (R^2 of Eq. A1) and their
    exact derivatives with respect to the centre and g1, written from that
    formula (float32, stamps back to back)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    pix, tx, tg1 = [], [], []
    for c0 in range(0, count, 5000):
        m = min(5000, count - c0)
        xc = (w / 2 + rng.uniform(-2, 2, m))[:, None, None]
        yc = (h / 2 + rng.uniform(-2, 2, m))[:, None, None]
        g1 = rng.uniform(-0.25, 0.25, m)[:, None, None]
        g2 = rng.uniform(-0.25, 0.25, m)[:, None, None]
        s = rng.uniform(2.0, 3.0, m)[:, None, None]
        t1, t2 = xx[None] - xc, yy[None] - yc
        A, B_ = (1 - g1) ** 2 + g2 ** 2, (1 + g1) ** 2 + g2 ** 2
        R2 = A * t1 * t1 + B_ * t2 * t2 - 4 * g2 * t1 * t2
        G = 100.0 * np.exp(-R2 / (2 * s * s))
        pix.append(G.astype(np.float32).ravel())
        tx.append((G * (2 * A * t1 - 4 * g2 * t2) / (2 * s * s)).astype(np.float32).ravel())
        tg1.append((-G * ((2 * g1 - 2) * t1 * t1 + (2 * g1 + 2) * t2 * t2) / (2 * s * s))
                   .astype(np.float32).ravel())
    return np.concatenate(pix), np.concatenate(tx), np.concatenate(tg1)


def test_moment_jvp_covariance_full_size(ctx):
    """At 100,000 stamps of 48x48 (the launch shape of the benchmark's
    workload): on noiseless elliptical Gaussians the GPU's own fixed point
    (matched weight) moves with the image, so the JVP along the exact
    derivative with respect to the centre is (1, 0, 0, 0, 0) and along g1 it is
    (0, 0, 1, 0, 0), to fp32 accuracy; and <v, JVP u> = <VJP v, u>."""
    n, h, w = 100_000, 48, 48
    pix, tx, tg1 = _gaussian_batch(n, h, w, seed=3)
    pix_d = torch.as_tensor(pix).cuda()
    idx = B.make_index(torch.arange(n, dtype=torch.int64).cuda() * h * w,
                       torch.full((n,), h, dtype=torch.int32).cuda(), torch.full((n,), w, dtype=torch.int32).cuda())
    opts = B.default_opts(max_pix=h * w, sigw_mode=0)
    mom = ctx.centroid(pix_d, idx, opts=opts)
    ctx.ellipticity(pix_d, idx, mom, opts=opts)
    r = B.results(mom)
    ok = (r["status"] & 1).astype(bool) & ~((r["status"] & ST["SIGW_CLAMPED"]).astype(bool))
    assert ok.mean() > 0.99
    mode = B.FSE_MOM_ELLIP
    dx = ctx.moment_jvp(pix_d, idx, mom, torch.as_tensor(tx).cuda(), mode=mode).cpu().numpy()[ok]
    dg = ctx.moment_jvp(pix_d, idx, mom, torch.as_tensor(tg1).cuda(), mode=mode).cpu().numpy()[ok]
    assert np.abs(dx - [1, 0, 0, 0, 0]).max() <= 2e-3, np.abs(dx - [1, 0, 0, 0, 0]).max(axis=0)
    assert np.abs(dg - [0, 0, 1, 0, 0]).max() <= 2e-3, np.abs(dg - [0, 0, 1, 0, 0]).max(axis=0)
    # duality on the full launch
    rng = np.random.default_rng(4)
    v = torch.as_tensor(rng.normal(size=(n, 5)).astype(np.float32)).cuda()
    u = torch.as_tensor(rng.normal(size=n * h * w).astype(np.float32)).cuda()
    jv = ctx.moment_jvp(pix_d, idx, mom, u, mode=mode)
    vj = ctx.moment_vjp(pix_d, idx, mom, v, mode=mode)
    lhs = (v.double() * jv.double()).sum(dim=1).cpu().numpy()
    rhs = (vj.double() * u.double()).view(n, h * w).sum(dim=1).cpu().numpy()
    scale = (vj.double().abs() * u.double().abs()).view(n, h * w).sum(dim=1).cpu().numpy()
    assert np.all(np.abs(lhs - rhs)[ok] <= 1e-5 * scale[ok] + 1e-6)


def test_moment_grad_autograd(ctx, O):
    """moment_shape: forward by fse_centroid + fse_ellipticity, backward by
    fse_moment_vjp.  The pixel gradient of a linear loss matches the oracle's
    VJP at the oracle's own fixed point; the two fixed points differ by the
    moment parity tolerance (1e-4 px, 1e-5 in g), which moves the gradient by
    well under 1e-3 of its largest entry."""
    from paper_1203_0571_gb300.autograd import moment_shape
    batch = synth.make_workload(0, count=64)
    rec = oracle_fixed_point(O, batch, 1)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    pix = b.pix.clone().requires_grad_(True)
    theta = moment_shape(pix, idx, ctx, opts=B.default_opts(max_pix=1024))
    wts = np.array([1.0, -0.5, 3.0, 2.0, 0.7])
    (theta * torch.as_tensor(wts, dtype=torch.float32).cuda()).sum().backward()
    g = pix.grad.cpu().numpy()
    checked = 0
    for i in range(batch.count):
        if not int(rec["status"][i]) & ST["MOM_CONVERGED"]:
            continue
        o = int(batch.offset[i])
        I = batch.stamp(i).astype(np.float32)
        dI, sing = O.moment_vjp(I, theta32(rec[i]), wts, mode=oracle_mode(O, B.FSE_MOM_ELLIP | B.FSE_MOM_SIGW_R50,
                                                                         rec[i]))
        if sing:
            continue
        gi = g[o:o + I.size].reshape(I.shape)
        assert np.abs(gi - dI).max() <= 1e-3 * np.abs(dI).max(), (i, np.abs(gi - dI).max() / np.abs(dI).max())
        checked += 1
    assert checked >= 0.9 * batch.count


def test_moment_grad_edge_cases(ctx):
    batch = synth.make_workload(0, count=6)
    b = batch.to("cuda")
    idx = B.make_index(b.offset, b.h, b.w)
    opts = B.default_opts(max_pix=1024)
    mom = ctx.centroid(b.pix, idx, opts=opts)
    ctx.ellipticity(b.pix, idx, mom, opts=opts)
    rec = B.results(mom).copy()
    rec["status"][1] = ST["MOM_MAXITER"]                  # not converged
    b.pix[int(batch.offset[2]) + 5] = float("nan")         # non-finite pixel
    moments = torch.as_tensor(rec.view(np.uint8).reshape(-1, 64)).cuda()
    st = torch.zeros(6, dtype=torch.int32, device="cuda")
    v = torch.ones((6, 5), device="cuda")
    dpix = ctx.moment_vjp(b.pix, idx, moments, v, status=st).cpu().numpy()
    st = st.cpu().numpy()
    assert st[1] == ST["MOM_FAILED"] and st[2] == ST["NONFINITE"], st
    for i in (1, 2):
        o = int(batch.offset[i])
        assert not np.any(dpix[o:o + 1024])
    assert all(st[i] == 0 for i in (0, 3, 4, 5)), st
    # mode bits that exclude each other, and unknown bits, are rejected
    for bad in (B.FSE_MOM_SIGW_FIXED | B.FSE_MOM_SIGW_R50, 8):
        with pytest.raises(B.FseError):
            ctx.moment_vjp(b.pix, idx, moments, v, mode=bad)
    # an empty batch is a no-op
    ctx.moment_jvp(b.pix, idx[:0], moments[:0], torch.zeros(0, device="cuda"))
