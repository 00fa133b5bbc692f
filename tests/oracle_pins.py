"""Pins that tie the FP64 oracle to facts outside itself.

Each pin takes an ``oracle.Oracle`` and raises AssertionError if the oracle
disagrees with what the paper or the mathematics fixes.  The pin tests run
them on the committed oracle; the mutation tests run them on copies with a
planted mistake and require that at least one pin fails.

Sources of truth used here: closed forms stated in the paper (Sec. 2 gain k,
Eq. 10 half-light b(n), Eq. 13 closed-form I0), library routines
(scipy.special.gammainc / gammaincinv, scipy.integrate.quad), exact symmetry
of sampled images, the published asymptotic series of b(n), brute-force
search, finite differences, and the chi^2 distribution of a correct fit.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
from scipy import integrate, special

from paper_1203_0571_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_facts.json")


def facts() -> dict:
    with open(GOLDEN) as f:
        return json.load(f)


def _gauss(h, w, xc, yc, g1, g2, s_R, I0=100.0):
    """Noiseless elliptical Gaussian exp(-R^2(g)/2 s_R^2) sampled at pixel centres."""
    # a Sérsic n = 0.5 profile is a Gaussian: b = ln 2, r = R/(1-|g|)
    re = s_R * math.sqrt(2 * math.log(2)) / (1 - math.hypot(g1, g2))
    return synth.single_stamp(h, w, n=0.5, re=re, g1=g1, g2=g2, xc=xc, yc=yc, I0=I0)


# ---------------------------------------------------------------- b(n), P(a,x)
def pin_gamma_p_library(O):
    """P(a, x) equals scipy.special.gammainc over the range the fit uses."""
    for a in (0.1, 0.4, 1.0, 2.5, 7.0, 20.0):
        for x in (1e-3, 0.1, 1.0, a, a + 1.5, 3 * a + 5, 60.0):
            got, want = O.gamma_p(a, x), special.gammainc(a, x)
            assert abs(got - want) <= 1e-13, (a, x, got, want)


def pin_sersic_b(O):
    """b(n) is the half-light constant of Eq. 10: b(0.5) = ln 2, the n = 1 and
    n = 1.5 closed forms of P, and P(2n, b(n)) = 1/2 by the library."""
    f = facts()
    assert abs(O.sersic_b(0.5) - f["sersic_b_half"]["value"]) <= 2e-16
    b = O.sersic_b(1.0)
    assert abs(1 - math.exp(-b) * (1 + b) - 0.5) <= 1e-15
    b = O.sersic_b(1.5)
    assert abs(1 - math.exp(-b) * (1 + b + b * b / 2) - 0.5) <= 1e-15
    for n in np.linspace(0.2, 10.0, 50):
        assert abs(special.gammainc(2 * n, O.sersic_b(n)) - 0.5) <= 1e-13, n


def pin_sersic_db(O):
    """b'(n): the published large-n series b = 2n - 1/3 + 4/(405 n) + 46/(25515 n^2)
    + 131/(1148175 n^3) - 2194697/(30690717750 n^4) ... (Ciotti & Bertin 1999) differentiated term by term, and a
    central difference of the library's inverse gamma at moderate n."""
    for n in (20.0, 40.0):
        series = (2 - 4 / (405 * n ** 2) - 92 / (25515 * n ** 3) - 393 / (1148175 * n ** 4)
                  + 4 * 2194697 / (30690717750 * n ** 5))
        assert abs(O.sersic_db(n) - series) <= 2e-9, (n, O.sersic_db(n), series)
    for n in (0.3, 0.7, 1.0, 2.0, 4.5):
        h = 1e-5
        fd = (special.gammaincinv(2 * (n + h), 0.5) - special.gammaincinv(2 * (n - h), 0.5)) / (2 * h)
        assert abs(O.sersic_db(n) - fd) <= 1e-7 * max(1.0, abs(fd)), (n, O.sersic_db(n), fd)


# ---------------------------------------------------------------- flux
def pin_flux_closed_form(O):
    """F = 2 pi n Gamma(2n) b^-2n I0 r_e^2 q equals the numerically integrated
    Eq. 10 profile over the plane (elliptical area element q 2 pi r dr)."""
    for (I0, re, n, gabs) in ((3.0, 2.0, 0.5, 0.0), (1.0, 4.0, 1.0, 0.3), (7.0, 3.0, 2.5, 0.6),
                              (2.0, 5.0, 4.0, 0.1), (1.0, 1.5, 8.0, 0.45)):
        b = special.gammaincinv(2 * n, 0.5)
        q = (1 - gabs) / (1 + gabs)
        # integrate in t = (r/r_e)^(1/n): r dr = r_e^2 n t^(2n-1) dt
        val, _ = integrate.quad(lambda t: t ** (2 * n - 1) * math.exp(-b * t), 0, np.inf,
                                epsabs=0, epsrel=1e-13, limit=200)
        want = 2 * math.pi * q * I0 * re * re * n * val
        got = O.sersic_flux(I0, re, n, gabs)
        assert abs(got / want - 1) <= 1e-9, (n, got, want)


def pin_flux_pixel_sum(O):
    """The closed-form flux equals the sum of a finely super-sampled stamp that
    holds essentially all of the light (n = 1, r_e = 4 px in 128 x 128)."""
    img = synth.single_stamp(128, 128, n=1.0, re=4.0, g1=0.2, g2=-0.15, xc=63.3, yc=64.1,
                             I0=10.0, supersample=8)
    got = O.sersic_flux(10.0, 4.0, 1.0, math.hypot(0.2, -0.15))
    assert abs(img.sum() / got - 1) <= 1e-4, (img.sum(), got)


# ---------------------------------------------------------------- moments
def pin_centroid_symmetric(O):
    """A point-symmetric sampled image has its weighted-centroid fixed point at the
    symmetry centre exactly, for any weight size and ellipticity (Sec. 2 fixed point
    sum I W theta = 0)."""
    rng = np.random.default_rng(5)
    for (n, re, g1, g2) in ((1.0, 3.0, 0.0, 0.0), (3.0, 5.0, 0.25, -0.3), (0.5, 2.5, -0.4, 0.1)):
        img = synth.single_stamp(64, 64, n=n, re=re, g1=g1, g2=g2, xc=31.5, yc=31.5, I0=1000.0)
        noise = rng.normal(size=img.shape)
        img = img + 0.5 * (noise + noise[::-1, ::-1])
        r = O.centroid(img)
        assert r["status"] & 1, r
        assert abs(r["x0"] - 31.5) <= 1e-10 and abs(r["y0"] - 31.5) <= 1e-10, r
        r = O.measure(img)
        assert r["status"] & 1, r
        assert abs(r["x0"] - 31.5) <= 1e-10 and abs(r["y0"] - 31.5) <= 1e-10, r


def pin_centroid_gain(O):
    """Sec. 2: one pass with a circular Gaussian weight of size s_w on a circular
    Gaussian of size s offset by (dx, dy) gives <x>/N = k dx with
    k = s_w^2/(s^2 + s_w^2); k = 0.5 when s = s_w; and the fixed gain 0.75 then
    shrinks the offset by a factor 3."""
    f = facts()
    for (s, sw) in ((4.0, 3.0), (3.0, 3.0), (2.5, 5.0)):
        img = _gauss(96, 96, 48.3, 47.6, 0.0, 0.0, s)
        st = O.moment_step(img, 48.0, 48.0, 0.0, 0.0, sw, k_gain=1.0, ellip=False)
        k = sw * sw / (s * s + sw * sw)
        assert abs(st["dx"] - 0.3 * k) <= 1e-10 and abs(st["dy"] + 0.4 * k) <= 1e-10, (st, k)
        if s == sw:
            assert abs(k - f["centroid_gain_matched"]["value"]) < 1e-15
            st = O.moment_step(img, 48.0, 48.0, 0.0, 0.0, sw, k_gain=0.75, ellip=False)
            left = (0.3 - st["dx"]) / 0.3
            assert abs(left - f["centroid_contraction_k075"]["value"]) <= 1e-9, left


def pin_centroid_newton_gain(O):
    """Sec. 2 says k can also be "determined iteratively"; the oracle's k_gain <= 0
    branch takes it from the moments, as a Newton step on sum I W theta = 0.  For
    an elliptical Gaussian profile exp(-R^2(theta - D; g)/2 s^2) under a weight
    exp(-R^2(theta; g)/2 s_w^2) of the same g (Eq. A1), the product is a Gaussian,
    so sum I W theta = N(D) k D with k = s_w^2/(s^2 + s_w^2) and
    N(D) proportional to exp(-R^2(D; g)/2 (s^2 + s_w^2)).  The Newton step is then
    D / (1 - R^2(D; g)/(s^2 + s_w^2)) (Sherman-Morrison on the rank-one Jacobian),
    for any g; the fixed gain would give k D instead."""
    for (s, sw, g1, g2) in ((4.0, 3.0, 0.0, 0.0), (3.0, 3.0, 0.2, -0.25), (2.5, 5.0, -0.3, 0.1),
                            (3.5, 2.0, 0.1, 0.35)):
        img = _gauss(96, 96, 48.3, 47.6, g1, g2, s)
        st = O.moment_step(img, 48.0, 48.0, g1, g2, sw, k_gain=0.0, ellip=False)
        gg = g1 * g1 + g2 * g2
        dx, dy = 0.3, -0.4
        R2 = (1 + gg - 2 * g1) * dx * dx + (1 + gg + 2 * g1) * dy * dy - 4 * g2 * dx * dy
        f = 1.0 / (1.0 - R2 / (s * s + sw * sw))
        assert st["ok"], st
        assert abs(st["dx"] - dx * f) <= 1e-10 and abs(st["dy"] - dy * f) <= 1e-10, (s, sw, g1, g2, st, f)


def pin_gain_independent_fixed_point(O):
    """The fixed point sum I W theta = 0 of Sec. 2 does not depend on the gain k:
    on noisy stamps the iteration with k determined from the moments (k_gain = 0)
    and with the paper's fixed k = 0.75 converge to the same centre and
    ellipticity, with fewer passes for the determined gain; the fixed gain of 1
    (Eqs. 5-6 with k = 1) reaches it as well."""
    batch = synth.make_workload(0, count=12)
    for i in range(batch.count):
        I = batch.stamp(i)
        ref = O.measure(I, opts=O.default_opts(k_gain=0.75))
        if not (ref["status"] & 1):
            continue
        for k in (0.0, 1.0):
            r = O.measure(I, opts=O.default_opts(k_gain=k))
            assert r["status"] & 1, (i, k, r)
            for key in ("x0", "y0", "e1", "e2"):
                assert abs(r[key] - ref[key]) <= 1e-9, (i, k, key, r[key], ref[key])
            if k == 0.0:
                assert r["it_mom"] <= ref["it_mom"], (i, r["it_mom"], ref["it_mom"])


def pin_ellipticity_exact(O):
    """For an elliptical profile f(R(g)) the weight W(R(g_w)) at g_w = g makes the
    product a sheared circular function, so e^obs = 2g/(1+g^2) = e_w and g is the
    fixed point of Eq. 9.  Checked on well-sampled elliptical Gaussians."""
    for (g1, g2, s_R, xc, yc) in ((0.3, -0.25, 7.0, 63.2, 64.7), (-0.5, 0.3, 4.0, 64.4, 63.1),
                                  (0.05, 0.02, 6.0, 62.9, 63.6)):
        img = _gauss(128, 128, xc, yc, g1, g2, s_R)
        r = O.measure(img)
        assert r["status"] & 1, r
        assert abs(r["x0"] - xc) <= 1e-9 and abs(r["y0"] - yc) <= 1e-9, r
        assert abs(r["e1"] - g1) <= 1e-9 and abs(r["e2"] - g2) <= 1e-9, r
        gg = g1 * g1 + g2 * g2
        st = O.moment_step(img, xc, yc, g1, g2, r["sigma_w"])
        assert abs(st["e1"] - 2 * g1 / (1 + gg)) <= 1e-12 and abs(st["e2"] - 2 * g2 / (1 + gg)) <= 1e-12


def pin_ellipticity_step_newton(O):
    """The step of Eq. 9 with P^SH from Eqs. A5-A6 plus B7-B14 is first-order exact:
    from g_w = g + d it returns -d up to O(d^2), and at g_w = 0 on a slightly sheared
    round profile it returns the shear (the KSB limit).  A dropped or mistyped term in
    the appendices leaves an O(1) relative error instead."""
    g = (0.3, -0.25)
    c = 63.5
    img = _gauss(128, 128, c, c, g[0], g[1], 7.0)
    errs = {}
    for d in (1e-3, 1e-4):
        worst = 0.0
        for dirn in ((1.0, 0.0), (0.0, 1.0), (0.6, -0.8)):
            st = O.moment_step(img, c, c, g[0] + d * dirn[0], g[1] + d * dirn[1], 6.5)
            err = math.hypot(st["dg1"] + d * dirn[0], st["dg2"] + d * dirn[1]) / d
            worst = max(worst, err)
        errs[d] = worst
    assert errs[1e-4] <= 3e-4, errs
    assert 5.0 <= errs[1e-3] / errs[1e-4] <= 20.0, errs
    for gam in (1e-4,):
        img2 = _gauss(128, 128, c, c, gam, -0.5 * gam, 7.0)
        st = O.moment_step(img2, c, c, 0.0, 0.0, 7.0)
        assert abs(st["dg1"] / gam - 1) <= 1e-6 and abs(st["dg2"] / (-0.5 * gam) - 1) <= 1e-6, st


def pin_matched_sigma_w(O):
    """Mode 0 (matched weight, Sec. 4.2.1): for an elliptical Gaussian of size s the
    rule sigma_w^2 = sum I W R^2 / sum I W converges to sigma_w = s."""
    for (g1, g2, s_R) in ((0.0, 0.0, 5.0), (0.2, 0.3, 6.0)):
        img = _gauss(128, 128, 63.7, 64.2, g1, g2, s_R)
        r = O.measure(img, opts=O.default_opts(sigw_mode=0))
        assert r["status"] & 1, r
        assert abs(r["sigma_w"] - s_R) <= 1e-9, r
        assert abs(r["e1"] - g1) <= 1e-9 and abs(r["e2"] - g2) <= 1e-9, r


def pin_stages_chain(O):
    """fse_centroid then fse_ellipticity reach the same fixed point as the single
    chain of Sec. 4.1 (the fixed point does not depend on the path)."""
    rng = np.random.default_rng(11)
    for (n, re, g1, g2) in ((1.5, 3.0, 0.2, 0.1), (3.0, 4.0, -0.3, 0.25)):
        img = synth.single_stamp(48, 48, n=n, re=re, g1=g1, g2=g2, xc=23.4, yc=24.3, I0=300.0)
        img = img + rng.normal(size=img.shape)
        full = O.measure(img)
        c = O.centroid(img)
        e = O.ellipticity(img, c["x0"], c["y0"], c["sigma_w"])
        for k in ("x0", "y0", "e1", "e2"):
            assert abs(full[k] - e[k]) <= 1e-9, (k, full[k], e[k])


# ---------------------------------------------------------------- fit
def pin_fit_noiseless(O):
    """A noiseless Eq. 10 stamp (rendered independently, scipy b(n)) fitted with the
    true centre and ellipticity returns the true (I0, r_e, n)."""
    for (n, re, g1, g2, I0) in ((0.6, 2.5, 0.1, 0.2, 500.0), (1.3, 6.0, -0.3, 0.1, 80.0),
                                (3.0, 4.0, 0.25, -0.35, 2e3), (5.5, 5.0, 0.0, 0.4, 1e4)):
        img = synth.single_stamp(48, 48, n=n, re=re, g1=g1, g2=g2, xc=23.3, yc=24.6, I0=I0)
        r = O.sersic_fit(img, 23.3, 24.6, g1, g2, re / 1.1774)
        assert r["status"] & 2, r
        for k, v in (("I0", I0), ("re", re), ("n", n)):
            assert abs(r[k] / v - 1) <= 1e-8, (k, r[k], v)


def pin_fit_gradient_fd(O):
    """The fit's J^T r is half the gradient of the oracle's own chi^2 (Eq. 11):
    central finite differences in FP64."""
    img = synth.single_stamp(32, 32, n=2.2, re=3.5, g1=0.2, g2=-0.1, xc=15.3, yc=16.2, I0=800.0,
                             noise_sigma=1.0, seed=3)
    p = np.array([700.0, 3.2, 2.5])
    chi2, g, H = O.fit_eval(img, 15.3, 16.2, 0.2, -0.1, p)
    for a in range(3):
        h = 1e-5 * p[a]
        pp, pm = p.copy(), p.copy()
        pp[a] += h
        pm[a] -= h
        fd = (O.fit_eval(img, 15.3, 16.2, 0.2, -0.1, pp)[0] - O.fit_eval(img, 15.3, 16.2, 0.2, -0.1, pm)[0]) / (2 * h)
        assert abs(2 * g[a] - fd) <= 1e-6 * abs(fd) + 1e-6, (a, 2 * g[a], fd)
    # J^T J diagonal is positive and Cauchy-Schwarz holds
    assert all(H[a, a] > 0 for a in range(3))
    assert H[0, 1] ** 2 <= H[0, 0] * H[1, 1] * (1 + 1e-12)


def pin_fit_minimum(O):
    """At the fit's optimum the gradient of chi^2 vanishes (so I0 is the closed form
    of Eq. 13), and no point of a brute-force (r_e, n) grid with I0 profiled has a
    lower chi^2 (tiny 12 x 12 stamps)."""
    rng = np.random.default_rng(2)
    for trial in range(3):
        n0, re0 = rng.uniform(0.8, 2.5), rng.uniform(1.5, 2.5)
        img = synth.single_stamp(12, 12, n=n0, re=re0, g1=0.1, g2=0.05, xc=5.6, yc=5.3, I0=400.0,
                                 noise_sigma=1.0, seed=20 + trial)
        r = O.sersic_fit(img, 5.6, 5.3, 0.1, 0.05, 1.6)
        assert r["status"] & 2, r
        p = np.array([r["I0"], r["re"], r["n"]])
        chi2, g, H = O.fit_eval(img, 5.6, 5.3, 0.1, 0.05, p)
        for a in range(3):
            assert abs(g[a]) <= 1e-7 * math.sqrt(H[a, a] * max(chi2, 1.0)), (a, g, H)
        best = np.inf
        for re_ in np.linspace(0.5 * p[1], 1.5 * p[1], 61):
            for n_ in np.linspace(max(0.2, 0.5 * p[2]), min(10.0, 1.5 * p[2]), 61):
                c1, g1_, H1 = O.fit_eval(img, 5.6, 5.3, 0.1, 0.05, [1.0, re_, n_])
                I0 = (H1[0, 0] - g1_[0]) / H1[0, 0]          # sum I E / sum E^2
                c = O.fit_eval(img, 5.6, 5.3, 0.1, 0.05, [I0, re_, n_])[0]
                best = min(best, c)
        assert r["chi2"] <= best * (1 + 1e-12), (r["chi2"], best)


def pin_fit_chi2_distribution(O):
    """With the exact model family and the true centre and ellipticity, chi^2_min
    follows chi^2 with N-3 degrees of freedom (noise sigma = 1)."""
    vals = []
    N = 24 * 24
    for s in range(120):
        img = synth.single_stamp(24, 24, n=1.5, re=3.0, g1=0.2, g2=0.1, xc=11.7, yc=12.2,
                                 I0=200.0, noise_sigma=1.0, seed=100 + s)
        r = O.sersic_fit(img, 11.7, 12.2, 0.2, 0.1, 2.2)
        vals.append(r["chi2"] / (N - 3))
    m = float(np.mean(vals))
    assert abs(m - 1.0) <= 4 * math.sqrt(2.0 / (N - 3)) / math.sqrt(len(vals)), m


def pin_r50_gaussian(O):
    """Start-up (Sec. 4.1): the growth-curve half-light radius of a circular
    Gaussian of size s centred on a pixel is s sqrt(2 ln 2) (half the flux of a
    2-D Gaussian lies inside that radius), up to pixelisation (< 3 %)."""
    for s_ in (2.0, 3.0, 4.0, 6.0, 8.0):
        img = _gauss(64, 64, 32.0, 32.0, 0.0, 0.0, s_)
        r = O.centroid(img)
        assert abs(r["r50"] / (math.sqrt(2 * math.log(2)) * s_) - 1) <= 0.03, (s_, r["r50"])


def _grad_case(k):
    rng = np.random.default_rng(40 + k)
    h, w = int(rng.integers(14, 30)), int(rng.integers(14, 30))
    n, re = rng.uniform(0.6, 6.0), rng.uniform(1.5, 4.0)
    g1, g2 = rng.uniform(-0.35, 0.35, 2)
    xc, yc = (w - 1) / 2 + rng.uniform(-1, 1), (h - 1) / 2 + rng.uniform(-1, 1)
    img = synth.single_stamp(h, w, n=n, re=re, g1=g1, g2=g2, xc=xc, yc=yc, I0=400.0,
                             noise_sigma=1.0, seed=60 + k)
    # evaluate away from the generating point so that the residuals are not pure noise
    p = np.array([xc + 0.07, yc - 0.05, g1 + 0.02, g2 - 0.015, 380.0, re * 1.05, n * 0.96])
    return img, p


def pin_chi2_grad_fd(O):
    """The analytic gradient of chi^2 (Eq. 11) with respect to (x0, y0, g1, g2, I0,
    r_e, n) and to a pixel equals Richardson-extrapolated central differences of
    chi^2; chi^2 itself equals the fit's evaluation of Eq. 11."""
    for k in range(4):
        img, p = _grad_case(k)
        iv = None if k % 2 == 0 else 0.5 + np.random.default_rng(k).random(img.shape)
        chi2, g, dpix = O.chi2_grad(img, p, ivar=iv, pixels=True)
        assert abs(chi2 / O.fit_eval(img, p[0], p[1], p[2], p[3], p[4:], ivar=iv)[0] - 1) <= 1e-12
        scale = np.array([1.0, 1.0, 0.1, 0.1, abs(p[4]), p[5], p[6]])
        for a in range(7):
            def f(hh):
                q = p.copy()
                q[a] += hh
                return O.chi2_grad(img, q, ivar=iv)[0]
            hs = 1e-3 * scale[a]
            d1 = (f(hs) - f(-hs)) / (2 * hs)
            d2 = (f(hs / 2) - f(-hs / 2)) / hs
            fd = (4 * d2 - d1) / 3
            assert abs(g[a] - fd) <= 1e-7 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, a, g[a], fd)
        i, j = img.shape[0] // 2, img.shape[1] // 3
        def fp(hh):
            im = img.copy()
            im[i, j] += hh
            return O.chi2_grad(im, p, ivar=iv)[0]
        fd = (fp(1e-3) - fp(-1e-3)) / 2e-3           # chi^2 is quadratic in a pixel: exact
        assert abs(dpix[i, j] - fd) <= 1e-6 * max(1.0, abs(fd)), (dpix[i, j], fd)


def pin_chi2_grad_noiseless(O):
    """A noiseless Eq. 10 stamp rendered independently (scipy's b(n)) has chi^2 = 0
    and a zero gradient at its generating parameters."""
    img = synth.single_stamp(26, 22, n=3.3, re=2.7, g1=-0.2, g2=0.3, xc=10.4, yc=12.9, I0=250.0)
    chi2, g = O.chi2_grad(img, [10.4, 12.9, -0.2, 0.3, 250.0, 2.7, 3.3])
    assert chi2 <= 1e-18 and np.abs(g).max() <= 1e-7, (chi2, g)


def pin_star_gaussian(O):
    """Sec. 4.2 Gaussian star: on a noiseless, well-sampled elliptical Gaussian
    the matched-weight iteration returns its sigma along the major axis and I0
    (Eqs. for sigma and I0 with s_w = s), and the flux closed form
    2 pi s^2 I0 q equals the pixel sum."""
    for s_, g1, g2 in ((2.3, 0.15, -0.1), (3.1, -0.2, 0.05), (2.0, 0.0, 0.0)):
        re = s_ * math.sqrt(2 * math.log(2))      # the n = 0.5 Sersic profile is this Gaussian
        img = synth.single_stamp(64, 64, n=0.5, re=re, g1=g1, g2=g2, xc=31.3, yc=32.6, I0=500.0)
        r = O.star(img, 31.3, 32.6, g1, g2, 1.5, "gauss")
        assert r["status"] & 1, r
        assert abs(r["size"] / s_ - 1) <= 1e-9 and abs(r["I0"] / 500.0 - 1) <= 1e-9, r
        assert abs(r["flux"] / img.sum() - 1) <= 1e-9, (r["flux"], img.sum())
        assert abs(r["r50"] - re) <= 1e-8 * re


def pin_star_moffat(O):
    """Sec. 4.2 Moffat star with the Moffat weight of exponent 3: on noiseless,
    well-sampled elliptical Moffat profiles (r_d 10-12 px, beta 4.5-5, so that
    pixelisation and the stamp edge are negligible) the iteration returns beta,
    r_d and I0; the flux closed form pi r_d^2 I0 q / (beta - 1) equals the pixel
    sum, and half of the flux of the profile lies inside
    r50 = r_d sqrt(2^(1/(beta-1)) - 1) (numerical integration)."""
    for beta, rd, g1, g2 in ((4.5, 10.0, 0.1, -0.05), (5.0, 12.0, 0.0, 0.2)):
        img = synth.moffat_stamp(128, 128, beta=beta, rd=rd, g1=g1, g2=g2, xc=63.4, yc=64.2, I0=300.0)
        r = O.star(img, 63.4, 64.2, g1, g2, 9.4, "moffat")
        assert r["status"] & 1, r
        assert abs(r["beta"] / beta - 1) <= 1e-5 and abs(r["size"] / rd - 1) <= 1e-5, r
        assert abs(r["I0"] / 300.0 - 1) <= 1e-5, r
        assert abs(r["flux"] / img.sum() - 1) <= 1e-5, (r["flux"], img.sum())
        b, d = r["beta"], r["size"]
        prof = lambda x: (1 + x * x / (d * d)) ** -b * 2 * math.pi * x
        tot = integrate.quad(prof, 0, np.inf)[0]
        half = integrate.quad(prof, 0, r["r50"])[0]
        assert abs(half / tot - 0.5) <= 1e-9, half / tot


def _ellip_gaussian(h, w, xc, yc, g1, g2, sig, amp):
    """amp exp(-R^2 / 2 sig^2) with R^2 of Eq. A1, and its derivatives with
    respect to the centre, g1, g2, sig and amp, written from that formula."""
    yy, xx = np.mgrid[0:h, 0:w].astype(float)
    t1, t2 = xx - xc, yy - yc
    A, B = (1 - g1) ** 2 + g2 ** 2, (1 + g1) ** 2 + g2 ** 2
    R2 = A * t1 * t1 + B * t2 * t2 - 4 * g2 * t1 * t2
    G = amp * np.exp(-R2 / (2 * sig * sig))
    k = G / (2 * sig * sig)
    tangents = [k * (2 * A * t1 - 4 * g2 * t2),                          # d/d xc
                k * (2 * B * t2 - 4 * g2 * t1),                          # d/d yc
                -k * ((2 * g1 - 2) * t1 * t1 + (2 * g1 + 2) * t2 * t2),  # d/d g1
                -k * (2 * g2 * (t1 * t1 + t2 * t2) - 4 * t1 * t2),       # d/d g2
                G * R2 / sig ** 3,                                       # d/d sig
                G / amp]                                                 # d/d amp
    return G, tangents


def _moment_theta(O, I, sigw_mode, ellip=True):
    """The oracle's moment fixed point (xc, yc, g1, g2, sigma_w), converged far
    below the differences taken from it."""
    o = O.default_opts(tol_pos=1e-13, tol_g=1e-13, tol_sig=1e-13, max_iter_mom=5000, sigw_mode=sigw_mode)
    r = O.centroid(I, o)
    if ellip:
        r = O.ellipticity(I, r["x0"], r["y0"], r["sigma_w"], o)
    assert r["status"] & 1, r
    return np.array([r["x0"], r["y0"], r["e1"] if ellip else 0.0, r["e2"] if ellip else 0.0, r["sigma_w"]])


def pin_moment_gradient_closed_forms(O):
    """Implicit gradients of the moment fixed point (Secs. 2-3), matched weight.
    On a well-sampled elliptical Gaussian the fixed point is its own centre, g
    and sigma (the weight then has the image's shape and sigma_w^2 =
    sum I W R^2 / sum I W = sigma^2), so it moves with the image: the derivative
    along the image's change of centre, g1, g2 or sigma is the unit vector of
    that parameter, and along its amplitude it is zero (the conditions are
    homogeneous in the pixels).  The fixed-point equations vanish there."""
    for xc, yc, g1, g2, sig in ((47.3, 48.6, 0.2, -0.15, 3.0), (40.8, 44.1, -0.1, 0.25, 3.4)):
        G, tangents = _ellip_gaussian(96, 96, xc, yc, g1, g2, sig, 100.0)
        th = _moment_theta(O, G, 0)
        assert np.allclose(th, [xc, yc, g1, g2, sig], atol=1e-9), th
        F, J = O.moment_jacobian(G, th)
        assert np.abs(F).max() <= 1e-9 * np.abs(J).max(), F
        for k, u in enumerate(tangents):
            d, singular = O.moment_jvp(G, th, u, mode=1)
            want = np.zeros(5)
            if k < 5:
                want[k] = 1.0
            assert not singular and np.abs(d - want).max() <= 1e-8, (k, d)


def pin_moment_gradient_fd(O):
    """Implicit gradients of the moment fixed point against central differences
    of the converged iteration itself, on a noisy stamp: Secs. 2-3 together and
    Sec. 2 alone, with the matched weight and with sigma_w from the growth-curve
    r50 (Sec. 4.1).  The VJP is the transpose of the JVP: <v, JVP u> = <VJP v, u>."""
    rng = np.random.default_rng(11)
    G, _ = _ellip_gaussian(64, 64, 31.6, 30.2, 0.18, 0.1, 3.0, 100.0)
    S = G + rng.normal(0.0, 0.5, G.shape)
    u = rng.normal(0.0, 1.0, G.shape)
    eps = 1e-4
    for sigw_mode, ellip in ((0, True), (1, True), (0, False), (1, False)):
        mode = (O.MOM_ELLIP if ellip else 0) | (O.MOM_SIGW_R50 if sigw_mode == 1 else 0)
        th = _moment_theta(O, S, sigw_mode, ellip)
        fd = (_moment_theta(O, S + eps * u, sigw_mode, ellip) -
              _moment_theta(O, S - eps * u, sigw_mode, ellip)) / (2 * eps)
        d, singular = O.moment_jvp(S, th, u, mode=mode)
        assert not singular and np.abs(d - fd).max() <= 1e-6 * np.abs(d).max(), (sigw_mode, ellip, d, fd)
        v = rng.normal(0.0, 1.0, 5)
        if not ellip:
            v[2:4] = 0.0
        dI, singular = O.moment_vjp(S, th, v, mode=mode)
        assert not singular and abs(v @ d - (dI * u).sum()) <= 1e-10 * np.abs(v).max() * np.abs(dI).sum()
    # J = dF/dtheta also away from the fixed point (where terms proportional to
    # F1, F2 no longer vanish): central differences of F in each parameter
    th = _moment_theta(O, S, 0) + np.array([0.3, -0.2, 0.05, -0.04, 0.2])
    _, J = O.moment_jacobian(S, th)
    for l in range(5):
        e = np.zeros(5)
        e[l] = 1e-5
        fd = (O.moment_jacobian(S, th + e)[0] - O.moment_jacobian(S, th - e)[0]) / 2e-5
        assert np.abs(J[:, l] - fd).max() <= 1e-6 * np.abs(J).max(), (l, J[:, l], fd)


def _growth_r50_bruteforce(I):
    """r50 by the rule of Sec. 4.1, restated with numpy: rings of integer
    radius k (k-1 < d <= k) around the brightest pixel (lowest row-major
    index on ties), summed outward until half the total; linear inside the
    crossing ring (k = 0: half the total over twice the peak)."""
    h, w = I.shape
    p = int(np.argmax(I.ravel()))          # first maximum in row-major order
    pr, pc = divmod(p, w)
    yy, xx = np.mgrid[0:h, 0:w]
    d2 = (yy - pr) ** 2 + (xx - pc) ** 2
    ring = np.ceil(np.sqrt(d2)).astype(int)
    sums = np.bincount(ring.ravel(), weights=I.ravel())
    enclosed = np.cumsum(sums)
    half = 0.5 * I.sum()
    k = int(np.argmax(enclosed >= half))
    if k == 0:
        return pr, pc, 0.5 * half / enclosed[0]
    return pr, pc, (k - 1) + (half - enclosed[k - 1]) / (enclosed[k] - enclosed[k - 1])


def pin_cutout(O):
    """The Sec. 4.1 cut-out: r50 equals a brute-force growth curve, the square
    of side 6 r50 (nearest integer) starts side/2 before the brightest pixel and
    is cut to the image; on a Gaussian it holds all but ~1e-3 of the flux;
    sides are clamped; non-finite images are refused."""
    rng = np.random.default_rng(21)
    for k in range(6):
        h, w = int(rng.integers(30, 90)), int(rng.integers(30, 90))
        yy, xx = np.mgrid[0:h, 0:w].astype(float)
        # the object inside, and near each corner, so that the square is cut
        xc, yc = [(rng.uniform(0, w - 1), rng.uniform(0, h - 1)), (w - 1.6, h - 2.2), (1.3, 0.8),
                  (w - 2.1, 1.4), (0.6, h - 1.3), (rng.uniform(0, w - 1), rng.uniform(0, h - 1))][k]
        sig = rng.uniform(1.0, 4.0)
        I = 200.0 * np.exp(-((xx - xc) ** 2 + (yy - yc) ** 2) / (2 * sig * sig)) + rng.normal(0, 0.3, (h, w))
        pr, pc, r50 = _growth_r50_bruteforce(I)
        c = O.cutout(I)
        assert abs(c["r50"] - r50) <= 1e-12 * max(1.0, r50), (k, c, r50)
        side = min(max(int(np.floor(6.0 * r50 + 0.5)), 8), 128)
        r0, c0 = pr - side // 2, pc - side // 2
        want = (max(r0, 0), max(c0, 0), min(r0 + side, h) - max(r0, 0), min(c0 + side, w) - max(c0, 0))
        assert (c["row0"], c["col0"], c["h"], c["w"]) == want, (k, c, want)
    # a well-sampled Gaussian: the square keeps all but about 1e-3 of its flux
    yy, xx = np.mgrid[0:256, 0:256].astype(float)
    G = np.exp(-((xx - 120.3) ** 2 + (yy - 131.7) ** 2) / (2 * 3.0 ** 2))
    c = O.cutout(G)
    inside = G[c["row0"]:c["row0"] + c["h"], c["col0"]:c["col0"] + c["w"]].sum() / G.sum()
    assert 0.998 <= inside < 1.0 and c["h"] == c["w"] == 21, (c, inside)
    # clamps and refusal
    assert O.cutout(G, side_factor=1.0)["h"] == 8 and O.cutout(G, side_factor=100.0)["h"] == 128
    bad = G.copy()
    bad[3, 4] = np.inf
    assert O.cutout(bad)["status"] & 16 and O.cutout(bad)["h"] == 0


def pin_fit_supersampled(O):
    """The pixel-integrated model (mean of S x S point samples per pixel): a
    noiseless stamp rendered independently with the same sub-grid (scipy's
    b(n)) is recovered exactly, with and without inverse variance, where the
    point-sampled fit on the same stamp is biased (small r_e, cuspy n); and
    its J^T r equals central differences of its chi^2."""
    rng = np.random.default_rng(8)
    for S, n, re, g1, g2 in ((4, 4.0, 1.2, 0.1, -0.15), (3, 1.0, 0.9, -0.2, 0.05), (2, 2.5, 1.6, 0.0, 0.3)):
        img = synth.single_stamp(32, 32, n=n, re=re, g1=g1, g2=g2, xc=15.3, yc=16.1, I0=500.0, supersample=S)
        iv = 0.5 + rng.random(img.shape)
        for ivar in (None, iv):
            r = O.sersic_fit(img, 15.3, 16.1, g1, g2, 1.5, ivar=ivar, opts=O.default_opts(supersample=S))
            assert r["status"] & 2, r
            assert abs(r["re"] / re - 1) <= 1e-8 and abs(r["n"] / n - 1) <= 1e-8, (S, r)
            assert abs(r["I0"] / 500.0 - 1) <= 1e-8 and r["chi2"] <= 1e-12, (S, r)
        r1 = O.sersic_fit(img, 15.3, 16.1, g1, g2, 1.5)
        assert abs(r1["n"] / n - 1) > 1e-3 or abs(r1["re"] / re - 1) > 1e-3, (S, r1)
        # gradient of the supersampled chi^2 against Richardson differences
        p = np.array([430.0, re * 1.07, n * 0.93])
        _, g, _ = O.fit_eval(img, 15.3, 16.1, g1, g2, p, supersample=S)
        for a in range(3):
            def f(hh):
                q = p.copy()
                q[a] += hh
                return O.fit_eval(img, 15.3, 16.1, g1, g2, q, supersample=S)[0]
            hs = 1e-4 * p[a]
            d1 = (f(hs) - f(-hs)) / (2 * hs)
            d2 = (f(hs / 2) - f(-hs / 2)) / hs
            fd = (4 * d2 - d1) / 3
            assert abs(2 * g[a] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(2 * g).max()), (S, a, 2 * g[a], fd)


def pin_edge_cases(O):
    """Status codes: non-finite pixels, empty flux, out-of-range sizes."""
    img = np.ones((8, 8))
    img[3, 4] = np.nan
    assert O.measure(img)["status"] & 16
    assert O.measure(np.zeros((8, 8)))["status"] & (2048 | 64)
    res, _ = O.batch(np.zeros(4, np.float32), [0], [0], [4])
    assert res["status"][0] & 32
    res, _ = O.batch(np.zeros(129 * 129, np.float32), [0], [129], [129])
    assert res["status"][0] & 32


ALL_PINS = [pin_gamma_p_library, pin_sersic_b, pin_sersic_db, pin_flux_closed_form,
            pin_flux_pixel_sum, pin_centroid_symmetric, pin_centroid_gain, pin_centroid_newton_gain,
            pin_gain_independent_fixed_point, pin_ellipticity_exact,
            pin_ellipticity_step_newton, pin_matched_sigma_w, pin_stages_chain, pin_fit_noiseless,
            pin_fit_gradient_fd, pin_fit_minimum, pin_fit_chi2_distribution, pin_r50_gaussian,
            pin_chi2_grad_fd, pin_chi2_grad_noiseless, pin_star_gaussian, pin_star_moffat,
            pin_moment_gradient_closed_forms, pin_moment_gradient_fd, pin_cutout, pin_fit_supersampled,
            pin_edge_cases]
