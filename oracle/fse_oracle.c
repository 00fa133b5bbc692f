/*
 * fse_oracle.c -- plain, slow FP64 reference of the fast shape estimator of
 * Li, Xin & Cui (2012), "Fast Shape Estimation for Galaxies and Stars".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this file.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA library; the two are written independently and
 * compared on the same seeded input stamps.
 *
 * Everything is double precision, one pixel at a time, in the order and
 * notation of the paper:
 *   - Sec. 2 (Eqs. 2-6): Gaussian-weighted first moments, centroid shift
 *     <x>/N = k dx with a fixed gain k = 0.75.
 *   - Sec. 3 (Eqs. 7-9) with Appendix A (Eqs. A1-A6) and Appendix B (Eqs.
 *     B7-B14): KSB shear polarisability with an elliptical weight and the
 *     iterative ellipticity update dg = (1-g_w^2) (P^SH)^-1 (e^obs - e_w).
 *   - Sec. 4.1 (Eqs. 10-13): Sérsic profile, chi^2, closed-form I0, and the
 *     profile fit with I0 profiled by Eq. 13 (the paper used MINUIT over (r_e, n);
 *     here Levenberg-Marquardt over (r_e, n)).
 *   - Sec. 4.1 start-up: brightest pixel and the half-light radius from the
 *     growth curve around it.
 *   - Sec. 4.2: Gaussian and Moffat star profiles from weighted radial moments.
 *   - Gradients: the chi^2 adjoint (Eqs. 10-12) and the implicit-function
 *     derivatives of the moment fixed point (Secs. 2-3) with respect to the
 *     pixels.
 *
 * Results are defined as converged fixed points / minima: the iterations run
 * to 1e-12 (moments) and 1e-10 (fit), far below the paper's 1e-4 stop, so that
 * any correct implementation converging to the same point agrees.
 *
 * Readings of points where the paper is silent or garbled (all listed in the
 * design notes):
 *   - W = exp(-R^2 / 2 sigma_w^2), R^2 from Eq. A1 (no normalisation), so the
 *     prime (derivative with respect to R^2) is W' = -W / (2 sigma_w^2).
 *   - T (undefined in the paper) is the weighted trace  sum f W theta^2.
 *   - e_w, "the ellipticity corresponding to g_w", is 2 g_w / (1 + |g_w|^2).
 *   - The symbols g_{s2} (Eq. A5) and g_1, g_2 inside Appendix B are read as
 *     the weight's g_w1, g_w2.
 *   - The centroid and ellipticity updates are taken from the same weighted
 *     pass (one pass per iteration) and applied together.
 *   - A step that would take |g_w| past (1 + |g_w|)/2 is shortened radially to
 *     that radius (|g| < 1 must hold; the first, circular-weight step can
 *     overshoot on very elliptical or cuspy objects).
 *   - sigma_w: mode 1 (default) keeps sigma_w = r50 / sqrt(2 ln 2) fixed; mode 0
 *     iterates the matched-weight rule sigma_w^2 = sum f W R^2 / sum f W of
 *     Sec. 4.2.1.  Both are clamped to [0.5, min(h,w)/2] px.
 *   - The Sérsic radius of an elliptical profile is r = R(g) / (1 - |g|), so
 *     r_e is the semi-major-axis half-light radius; q = (1-|g|)/(1+|g|).
 *   - b(n) is the exact root of P(2n, b) = 1/2 (regularised lower incomplete
 *     gamma), so that r_e is the half-light radius as Eq. 10 requires.
 *   - The model is sampled at pixel centres.
 *
 * Parity is pinned (see tests) by closed forms: the exact centroid of a
 * point-symmetric stamp, the one-step Gaussian gain k = s_w^2/(s^2+s_w^2),
 * the exact ellipticity of an elliptical Gaussian, the matched sigma_w of a
 * Gaussian, b(0.5) = ln 2 and the n = 1 identity, P(2n, b(n)) = 1/2 against a
 * library routine, the flux closed form against a super-sampled pixel sum,
 * the exact recovery of a noiseless Sérsic stamp, a brute-force (r_e, n) grid
 * on tiny stamps, and central finite differences for the gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Types (the oracle's own; the Python harness converts).                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double tol_pos;      /* centroid step stop, px                       */
    double tol_g;        /* ellipticity step stop                        */
    double tol_sig;      /* relative sigma_w step stop (mode 0)          */
    double tol_fit;      /* relative parameter step stop of the fit      */
    int    max_iter_mom;
    int    max_iter_fit;
    double k_gain;       /* Sec. 2: 0.75                                 */
    int    sigw_mode;    /* 0 adaptive matched, 1 fixed from r50         */
    double n_min, n_max; /* fit bounds on n                              */
    double re_min;       /* lower bound on r_e, px                       */
    double re_max_frac;  /* upper bound on r_e = re_max_frac * max(h,w)  */
    double lm_lambda0;
    int    supersample;  /* S: the model of a pixel is the mean of S x S point
                            samples on a regular sub-grid (1: the pixel centre) */
} orc_opts;

typedef struct {
    double x0, y0, e1, e2, sigma_w, r50;
    double I0, re, n, flux, chi2;
    int32_t npix, it_mom, it_fit;
    uint32_t status;
} orc_result;

/* status bits (the oracle's own numbering, mirrored by value in the ABI) */
#define ORC_MOM_CONVERGED   (1u << 0)
#define ORC_FIT_CONVERGED   (1u << 1)
#define ORC_MOM_MAXITER     (1u << 2)
#define ORC_FIT_MAXITER     (1u << 3)
#define ORC_NONFINITE       (1u << 4)
#define ORC_BAD_SIZE        (1u << 5)
#define ORC_MOM_FAILED      (1u << 6)
#define ORC_FIT_BOUND       (1u << 7)
#define ORC_FIT_SINGULAR    (1u << 8)
#define ORC_NONPOS_FLUX     (1u << 9)
#define ORC_SIGW_CLAMPED    (1u << 10)
#define ORC_INIT_FALLBACK   (1u << 11)

#define SQRT_2LN2 1.1774100225154747   /* half-light radius / sigma of a Gaussian */

void orc_default_opts(orc_opts *o)
{
    o->tol_pos = 1e-12;
    o->tol_g = 1e-12;
    o->tol_sig = 1e-12;
    o->tol_fit = 1e-10;
    o->max_iter_mom = 500;
    o->max_iter_fit = 200;
    o->k_gain = 0.75;
    o->sigw_mode = 1;
    o->n_min = 0.2;
    o->n_max = 10.0;
    o->re_min = 0.2;
    o->re_max_frac = 2.0;
    o->lm_lambda0 = 1e-3;
    o->supersample = 1;
}

/* ------------------------------------------------------------------------ */
/* Regularised lower incomplete gamma P(a, x) and the Sérsic b(n).           */
/* Series (Abramowitz & Stegun 6.5.29) for x < a + 1, Legendre continued      */
/* fraction for Q = 1 - P (A&S 6.5.31, evaluated by the modified Lentz       */
/* method) otherwise -- the standard published scheme (Numerical Recipes     */
/* Sec. 6.2).                                                                */
/* ------------------------------------------------------------------------ */
double orc_gamma_p(double a, double x)
{
    if (x <= 0.0) return 0.0;
    double lpre = a * log(x) - x - lgamma(a);
    if (x < a + 1.0) {
        /* P = x^a e^-x / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)) */
        double term = 1.0 / a, sum = term;
        for (int k = 1; k < 100000; ++k) {
            term *= x / (a + k);
            sum += term;
            if (fabs(term) < fabs(sum) * 1e-17) break;
        }
        return sum * exp(lpre);
    }
    /* Q = x^a e^-x / Gamma(a) * 1/(x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(x+5-a- ...))) */
    const double tiny = 1e-300;
    double bb = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / bb, h = d;
    for (int i = 1; i < 100000; ++i) {
        double an = -i * (i - a);
        bb += 2.0;
        d = an * d + bb;
        if (fabs(d) < tiny) d = tiny;
        c = bb + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        double del = d * c;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return 1.0 - exp(lpre) * h;
}

/* b(n): the root of P(2n, b) = 1/2, i.e. the constant that makes r_e the
 * half-light radius of I(r) = I0 exp(-b (r/r_e)^(1/n))  (Eq. 10).
 * Newton on P with dP/db = b^(a-1) e^-b / Gamma(a), safeguarded by bisection
 * on the bracket (0, a]: the median of a Gamma(a) variable lies below its
 * mean a. */
double orc_sersic_b(double n)
{
    double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = a - 1.0 / 3.0;
    if (b <= lo || b >= hi) b = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = orc_gamma_p(a, b) - 0.5;
        if (f > 0.0) hi = b; else lo = b;
        double fp = exp((a - 1.0) * log(b) - b - lgamma(a));
        double nb = b - f / fp;
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        if (fabs(nb - b) <= 1e-16 * fabs(b) || hi - lo <= 1e-16 * hi) { b = nb; break; }
        b = nb;
    }
    return b;
}

/* b'(n) by a Richardson-extrapolated central difference of b(n). */
double orc_sersic_db(double n)
{
    double h = 1e-3 * (n > 1.0 ? n : 1.0);
    if (n - h < 0.05) h = 0.5 * (n - 0.05);
    double d1 = (orc_sersic_b(n + h) - orc_sersic_b(n - h)) / (2.0 * h);
    double d2 = (orc_sersic_b(n + 0.5 * h) - orc_sersic_b(n - 0.5 * h)) / h;
    return (4.0 * d2 - d1) / 3.0;
}

/* Total flux of the elliptical Sérsic profile (integral of Eq. 10 over the
 * plane, elliptical area element q 2 pi r dr):
 *   F = 2 pi n Gamma(2n) b^-2n I0 r_e^2 q,  q = (1-|g|)/(1+|g|). */
double orc_sersic_flux(double I0, double re, double n, double gabs)
{
    double b = orc_sersic_b(n);
    double q = (1.0 - gabs) / (1.0 + gabs);
    return 2.0 * M_PI * n * exp(lgamma(2.0 * n) - 2.0 * n * log(b)) * I0 * re * re * q;
}

/* ------------------------------------------------------------------------ */
/* Elliptical weight metric, Eq. A1.                                         */
/* ------------------------------------------------------------------------ */
static double ellip_R2(double t1, double t2, double g1, double g2)
{
    return ((1.0 - g1) * (1.0 - g1) + g2 * g2) * t1 * t1
         + ((1.0 + g1) * (1.0 + g1) + g2 * g2) * t2 * t2
         - 4.0 * g2 * t1 * t2;
}

/* ------------------------------------------------------------------------ */
/* Start-up (Sec. 4.1): brightest pixel, total, growth-curve r50.            */
/* ------------------------------------------------------------------------ */
static int init_stamp_k(const double *I, int h, int w, int *pk_row, int *pk_col,
                        double *r50, uint32_t *status, int *k_cross);

static int init_stamp(const double *I, int h, int w, int *pk_row, int *pk_col,
                      double *r50, uint32_t *status)
{
    return init_stamp_k(I, h, w, pk_row, pk_col, r50, status, NULL);
}

/* As init_stamp; *k_cross (if not NULL) receives the ring in which the growth
 * curve crosses half the total, or -1 for the fallback radius. */
static int init_stamp_k(const double *I, int h, int w, int *pk_row, int *pk_col,
                        double *r50, uint32_t *status, int *k_cross)
{
    if (k_cross) *k_cross = -1;
    int npix = h * w, best = 0;
    for (int p = 0; p < npix; ++p) {
        if (!isfinite(I[p])) { *status |= ORC_NONFINITE; return 0; }
        if (I[p] > I[best]) best = p;           /* ties keep the lowest index */
    }
    *pk_row = best / w;
    *pk_col = best % w;
    double total = 0.0;
    for (int p = 0; p < npix; ++p) total += I[p];
    if (!(total > 0.0)) { *status |= ORC_INIT_FALLBACK; *r50 = SQRT_2LN2; return 1; }
    /* Growth curve: pixels summed outward from the brightest one, in rings
     * of integer radius k (pixels with k-1 < d <= k), until the enclosed flux
     * reaches half of the stamp total; r50 interpolates linearly inside the
     * ring that crosses. */
    double half = 0.5 * total, prev = 0.0;
    int kmax = (int)ceil(sqrt((double)(h - 1) * (h - 1) + (double)(w - 1) * (w - 1))) + 1;
    for (int k = 0; k <= kmax; ++k) {
        double S = 0.0;
        for (int i = 0; i < h; ++i)
            for (int j = 0; j < w; ++j) {
                int di = i - *pk_row, dj = j - *pk_col;
                if (di * di + dj * dj <= k * k) S += I[i * w + j];
            }
        if (S >= half) {
            if (k_cross) *k_cross = k;
            if (k == 0) *r50 = 0.5 * half / S;
            else        *r50 = (k - 1) + (half - prev) / (S - prev);
            return 1;
        }
        prev = S;
    }
    *status |= ORC_INIT_FALLBACK;
    *r50 = SQRT_2LN2;
    return 1;
}

static double clamp_sigw(double s, int h, int w, uint32_t *status)
{
    double smax = 0.5 * (h < w ? h : w);
    if (s < 0.5) { *status |= ORC_SIGW_CLAMPED; return 0.5; }
    if (s > smax) { *status |= ORC_SIGW_CLAMPED; return smax; }
    return s;
}

/* ------------------------------------------------------------------------ */
/* One weighted pass and the moment updates.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    double dx, dy;      /* centroid step, Eqs. 5-6 with k = k_gain       */
    double dg1, dg2;    /* ellipticity step, Eq. 9                        */
    double sigw_new;    /* matched-weight rule (mode 0)                   */
    double e1, e2;      /* e^obs                                          */
    int ok;
} moment_step;

/* One pass over the stamp with weight W(R^2(g_w)) centred at (xc, yc).
 * If `ellip` is 0 only the centroid step (Sec. 2, circular weight) is formed. */
static moment_step weighted_pass(const double *I, int h, int w, double xc, double yc,
                                 double gw1, double gw2, double sw, double k_gain, int ellip)
{
    moment_step s;
    memset(&s, 0, sizeof s);
    double c = 1.0 / (2.0 * sw * sw);
    double gg = gw1 * gw1 + gw2 * gw2;
    double A = 1.0 + gg - 2.0 * gw1;        /* Appendix A */
    double B = 1.0 + gg + 2.0 * gw1;
    double N = 0, mx = 0, my = 0, Q11 = 0, Q22 = 0, Q12 = 0, SWR2 = 0;
    /* integrals of Appendix A */
    double X11 = 0, X12 = 0, X21 = 0, X22 = 0, eS1 = 0, eS2 = 0;
    /* integrals of Appendix B: sum f P_k */
    double P1 = 0, P2 = 0, P3 = 0, P4 = 0, P5 = 0, P6 = 0;
    for (int i = 0; i < h; ++i) {
        for (int j = 0; j < w; ++j) {
            double f = I[i * w + j];
            double t1 = j - xc, t2 = i - yc;
            double R2 = ellip_R2(t1, t2, gw1, gw2);
            double W = exp(-R2 * c);
            double Wp = -c * W;                       /* dW/dR^2 */
            N += f * W;                               /* Eq. 2 */
            mx += f * W * t1;                         /* Eq. 3 */
            my += f * W * t2;                         /* Eq. 4 */
            Q11 += f * W * t1 * t1;
            Q22 += f * W * t2 * t2;
            Q12 += f * W * t1 * t2;
            SWR2 += f * W * R2;
            if (!ellip) continue;
            double th2 = t1 * t1 + t2 * t2;
            double d1 = t1 * t1 - t2 * t2;            /* theta_1^2 - theta_2^2 */
            double p12 = t1 * t2;
            double a1 = A * t1 * t1 - B * t2 * t2;    /* Eq. A5-A6 brackets */
            double a2 = (A + B) * p12 - 2.0 * gw2 * th2;
            /* Eq. A5, X^SH integrands */
            X11 += f * (2.0 * W * th2 + 2.0 * Wp * d1 * a1);
            X12 += f * (2.0 * Wp * d1 * a2);
            X21 += f * (4.0 * Wp * p12 * a1);
            X22 += f * (2.0 * W * th2 + 4.0 * Wp * p12 * a2);
            /* Eq. A6, e^SH integrand */
            eS1 += f * Wp * th2 * a1;
            eS2 += f * Wp * th2 * a2;
            /* Eqs. B9-B14: P_1 ... P_6 */
            double b1 = A * t1 * t1 + B * t2 * t2 - 4.0 * gw2 * p12;
            double b2 = (A - B) * p12 + 2.0 * gw2 * d1;
            P1 += f * (4.0 * W * d1 + 2.0 * Wp * d1 * b1);
            P2 += f * (4.0 * W * p12 + 2.0 * Wp * d1 * b2);
            P3 += f * (8.0 * W * p12 + 4.0 * Wp * p12 * b1);
            P4 += f * (-2.0 * W * d1 + 4.0 * Wp * p12 * b2);
            P5 += f * (4.0 * W * th2 + 2.0 * Wp * th2 * b1);
            P6 += f * (2.0 * Wp * th2 * b2);
        }
    }
    if (!(N > 0.0)) return s;
    if (k_gain > 0.0) {
        s.dx = mx / (k_gain * N);                 /* Eqs. 5-6: <x>/N = k dx */
        s.dy = my / (k_gain * N);
    } else {
        /* k "determined iteratively" (Sec. 2): Newton on (<x>, <y>) = 0 with the
         * derivative of the weighted first moments with respect to the centre,
         * d<x>/dx_c = sum I [dW/dx_c theta_1 - W], dW/dx_c = 2 c W (A t1 - 2 g2 t2). */
        double J11 = 2.0 * c * (A * Q11 - 2.0 * gw2 * Q12) - N;
        double J12 = 2.0 * c * (B * Q12 - 2.0 * gw2 * Q11);
        double J21 = 2.0 * c * (A * Q12 - 2.0 * gw2 * Q22);
        double J22 = 2.0 * c * (B * Q22 - 2.0 * gw2 * Q12) - N;
        double dj = J11 * J22 - J12 * J21;
        if (!(dj > 0.0)) return s;
        s.dx = -(J22 * mx - J12 * my) / dj;
        s.dy = -(-J21 * mx + J11 * my) / dj;
    }
    s.sigw_new = SWR2 > 0.0 ? sqrt(SWR2 / N) : 0.0;
    if (!ellip) { s.ok = 1; return s; }
    double T = Q11 + Q22;
    if (!(T > 0.0)) return s;
    double e1 = (Q11 - Q22) / T, e2 = 2.0 * Q12 / T;
    s.e1 = e1; s.e2 = e2;
    /* X^SH (Eq. A5) plus Delta X^SH (Eq. B7) */
    double X[2][2] = {
        { X11 / T + (-gw1 * P1 - gw2 * P2) / T, X12 / T + (gw1 * P2 - gw2 * P1) / T },
        { X21 / T + (-gw1 * P3 - gw2 * P4) / T, X22 / T + (gw1 * P4 - gw2 * P3) / T } };
    /* e^SH (Eq. A6) plus Delta e^SH (Eq. B8) */
    double eSH[2] = { 2.0 * e1 + 2.0 * eS1 / T + (-gw1 * P5 - gw2 * P6) / T,
                      2.0 * e2 + 2.0 * eS2 / T + (gw1 * P6 - gw2 * P5) / T };
    /* Eq. 8: P^SH_ab = X^SH_ab - e_a e^SH_b */
    double P[2][2] = { { X[0][0] - e1 * eSH[0], X[0][1] - e1 * eSH[1] },
                       { X[1][0] - e2 * eSH[0], X[1][1] - e2 * eSH[1] } };
    double det = P[0][0] * P[1][1] - P[0][1] * P[1][0];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return s;
    /* Eq. 9: dg = (1 - g_w^2) P^-1 (e^obs - e_w), e_w = 2 g_w / (1 + g_w^2) */
    double r1 = e1 - 2.0 * gw1 / (1.0 + gg);
    double r2 = e2 - 2.0 * gw2 / (1.0 + gg);
    double s1 = (P[1][1] * r1 - P[0][1] * r2) / det;
    double s2 = (-P[1][0] * r1 + P[0][0] * r2) / det;
    s.dg1 = (1.0 - gg) * s1;
    s.dg2 = (1.0 - gg) * s2;
    s.ok = isfinite(s.dg1) && isfinite(s.dg2);
    return s;
}

/* Iterate to the fixed point.  ellip = 0: Sec. 2 centroid only (g_w = 0);
 * ellip = 1: centroid and ellipticity together (Secs. 2-3, Sec. 4.1). */
static void moment_iterate(const double *I, int h, int w, const orc_opts *o, int ellip,
                           double *xc, double *yc, double *g1, double *g2, double *sw,
                           int *iters, uint32_t *status)
{
    int it;
    for (it = 1; it <= o->max_iter_mom; ++it) {
        moment_step s = weighted_pass(I, h, w, *xc, *yc, *g1, *g2, *sw, o->k_gain, ellip);
        if (!s.ok) { *status |= ORC_MOM_FAILED; break; }
        *xc += s.dx;
        *yc += s.dy;
        double dsig = 0.0;
        if (ellip) {
            /* |g| < 1 must hold; a step that would take |g_w| past half-way to
             * the unit circle is shortened radially to (1 + |g_w|)/2. */
            double cap = 0.5 * (1.0 + sqrt(*g1 * *g1 + *g2 * *g2));
            double n1 = *g1 + s.dg1, n2 = *g2 + s.dg2, nn = sqrt(n1 * n1 + n2 * n2);
            if (nn > cap) { n1 *= cap / nn; n2 *= cap / nn; }
            *g1 = n1;
            *g2 = n2;
        }
        if (o->sigw_mode == 0) {
            double ns = clamp_sigw(s.sigw_new, h, w, status);
            dsig = fabs(ns - *sw) / *sw;
            *sw = ns;
        }
        if (*g1 * *g1 + *g2 * *g2 >= 0.95 * 0.95 ||
            *xc < -0.5 || *xc > w - 0.5 || *yc < -0.5 || *yc > h - 0.5) {
            *status |= ORC_MOM_FAILED;
            break;
        }
        if (fabs(s.dx) <= o->tol_pos && fabs(s.dy) <= o->tol_pos &&
            fabs(s.dg1) <= o->tol_g && fabs(s.dg2) <= o->tol_g && dsig <= o->tol_sig) {
            *status |= ORC_MOM_CONVERGED;
            break;
        }
    }
    if (it > o->max_iter_mom) { *status |= ORC_MOM_MAXITER; it = o->max_iter_mom; }
    *iters = it;
}

/* ------------------------------------------------------------------------ */
/* Sérsic fit (Sec. 4.1, Eqs. 10-13).                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *I, *ivar;
    const double *r;      /* Sérsic radius R(g)/(1-|g|) of each point sample,
                             ns per pixel (pixel i: r[i*ns ... i*ns + ns-1]) */
    int npix, ns;
} fit_data;

/* Sérsic radii of the point samples of every pixel: with supersample S the
 * S x S sub-grid points (j + (a + 1/2)/S - 1/2, i + (c + 1/2)/S - 1/2) of
 * pixel (i, j), S = 1 the pixel centre (Sec. 4.1 samples the profile at the
 * pixels; the mean over a finer grid approaches the pixel integral that
 * pixelation calls for, Sec. 4.2). */
static double *sample_radii(int h, int w, int S, double xc, double yc, double g1, double g2)
{
    double gabs = sqrt(g1 * g1 + g2 * g2);
    double *r = (double *)malloc(sizeof(double) * h * w * S * S);
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j)
            for (int c = 0; c < S; ++c)
                for (int a = 0; a < S; ++a) {
                    double oy = (c + 0.5) / S - 0.5, ox = (a + 0.5) / S - 0.5;
                    double R2 = ellip_R2(j + ox - xc, i + oy - yc, g1, g2);
                    r[((i * w + j) * S + c) * S + a] = sqrt(R2 > 0.0 ? R2 : 0.0) / (1.0 - gabs);
                }
    return r;
}

/* chi^2 (Eq. 11) and, if H != NULL, the normal equations J^T W J, J^T W r
 * of the model m = I0 exp(-b (r/r_e)^(1/n)) with respect to (I0, r_e, n).
 * A pixel's model and derivatives are the means over its point samples. */
static double fit_eval(const fit_data *d, const double p[3], double H[3][3], double g[3])
{
    double I0 = p[0], re = p[1], n = p[2];
    double b = orc_sersic_b(n), db = H ? orc_sersic_db(n) : 0.0;
    double chi2 = 0.0;
    if (H) { memset(H, 0, 9 * sizeof(double)); memset(g, 0, 3 * sizeof(double)); }
    for (int i = 0; i < d->npix; ++i) {
        double wgt = d->ivar ? d->ivar[i] : 1.0;
        double E = 0.0, J[3] = { 0.0, 0.0, 0.0 };
        for (int k = 0; k < d->ns; ++k) {
            double x = d->r[i * d->ns + k] / re;
            double u = x > 0.0 ? pow(x, 1.0 / n) : 0.0;
            double Ek = exp(-b * u);
            E += Ek;
            J[1] += I0 * Ek * b * u / (n * re);                              /* dm/dr_e */
            if (x > 0.0) J[2] += I0 * Ek * u * (b * log(x) / (n * n) - db);   /* dm/dn */
        }
        E /= d->ns;
        J[0] = E;                                                             /* dm/dI0 */
        J[1] /= d->ns;
        J[2] /= d->ns;
        double m = I0 * E;
        double res = m - d->I[i];
        chi2 += wgt * res * res;
        if (!H) continue;
        for (int a = 0; a < 3; ++a) {
            g[a] += wgt * J[a] * res;
            for (int c = 0; c < 3; ++c) H[a][c] += wgt * J[a] * J[c];
        }
    }
    return chi2;
}

/* The profiled problem of Sec. 4.1: for fixed (r_e, n) the amplitude is the
 * closed form of Eq. 13, I0 = sum I f / sum f^2 (weights 1/sigma_i^2), leaving
 * chi^2 a function of (r_e, n) alone.  Returns chi^2 at that I0 and, if Hr is
 * not NULL, the Gauss-Newton normal equations of the profiled residual
 * r_i = I0 f_i - I_i with the Jacobian (I - P_f) I0 df/dtheta (the derivative
 * of r with respect to (r_e, n) when I0 follows Eq. 13, dropping the term
 * proportional to the residual): gr = J^T W r, Hr = J^T W J. */
static double profiled_eval(const fit_data *d, double re, double n, double *I0_out,
                            double Hr[2][2], double gr[2])
{
    double b = orc_sersic_b(n);
    double sIf = 0.0, sff = 0.0;
    for (int i = 0; i < d->npix; ++i) {
        double wgt = d->ivar ? d->ivar[i] : 1.0;
        double f = 0.0;
        for (int k = 0; k < d->ns; ++k) {
            double x = d->r[i * d->ns + k] / re;
            f += exp(-b * (x > 0.0 ? pow(x, 1.0 / n) : 0.0));
        }
        f /= d->ns;
        sIf += wgt * d->I[i] * f;
        sff += wgt * f * f;
    }
    double I0 = sIf / sff;                                   /* Eq. 13 */
    *I0_out = I0;
    double p[3] = { I0, re, n }, H[3][3], g[3];
    double chi2 = fit_eval(d, p, Hr ? H : NULL, g);
    if (Hr) {
        /* eliminate I0: Schur complement of the I0 row/column of J^T W J */
        for (int a = 0; a < 2; ++a) {
            gr[a] = g[1 + a] - H[1 + a][0] * g[0] / H[0][0];
            for (int c = 0; c < 2; ++c)
                Hr[a][c] = H[1 + a][1 + c] - H[1 + a][0] * H[0][1 + c] / H[0][0];
        }
    }
    return chi2;
}

/* Keep (r_e, n) inside the fit's box. */
static void clamp_theta(double q[2], const orc_opts *o, double re_max)
{
    if (q[0] < o->re_min) q[0] = o->re_min;
    if (q[0] > re_max) q[0] = re_max;
    if (q[1] < o->n_min) q[1] = o->n_min;
    if (q[1] > o->n_max) q[1] = o->n_max;
}

/* Relative size max_i |s_i| / theta_i of the undamped Gauss-Newton step
 * s = -H^-1 g, clipped to the box (0 when the box stops it entirely); +inf
 * when H is not positive definite. */
static double gn_step(double H[2][2], const double g[2], const double th[2], const orc_opts *o,
                      double re_max)
{
    double det = H[0][0] * H[1][1] - H[0][1] * H[1][0];
    if (!(det > 0.0) || !(H[0][0] > 0.0) || !isfinite(det)) return INFINITY;
    double q[2] = { th[0] + (-H[1][1] * g[0] + H[0][1] * g[1]) / det,
                    th[1] + (H[1][0] * g[0] - H[0][0] * g[1]) / det };
    clamp_theta(q, o, re_max);
    return fmax(fabs(q[0] - th[0]) / th[0], fabs(q[1] - th[1]) / th[1]);
}

/* start (may be NULL): (r_e, n) to start the iteration from instead of the
 * Sec. 4.1 start below; used to test whether a lower chi^2 found elsewhere is
 * another local minimum of the same profiled problem. */
static void fit_stamp(const double *I, const double *ivar, int h, int w, const orc_opts *o,
                      double xc, double yc, double g1, double g2, double sw,
                      orc_result *res, const double *start)
{
    int npix = h * w;
    double gabs = sqrt(g1 * g1 + g2 * g2);
    int S = o->supersample > 1 ? o->supersample : 1;
    double *r = sample_radii(h, w, S, xc, yc, g1, g2);
    fit_data d = { I, ivar, r, npix, S * S };
    double re_max = o->re_max_frac * (h > w ? h : w);
    /* Start: r_e from the weight size, n the best of {0.5, 1, 2, 4}. */
    double re0 = SQRT_2LN2 * sw / (1.0 - gabs);
    if (re0 < o->re_min) re0 = o->re_min;
    if (re0 > re_max) re0 = re_max;
    const double n_start[4] = { 0.5, 1.0, 2.0, 4.0 };
    double th[2] = { re0, 1.0 }, I0 = 0.0, best = INFINITY;
    for (int c = 0; c < 4; ++c) {
        double I0c, chi2c = profiled_eval(&d, re0, n_start[c], &I0c, NULL, NULL);
        if (chi2c < best) { best = chi2c; th[1] = n_start[c]; }
    }
    if (start) { th[0] = start[0]; th[1] = start[1]; clamp_theta(th, o, re_max); }
    /* Levenberg-Marquardt on theta = (r_e, n) (the paper used MINUIT), with
     * the gain-ratio damping update of Nielsen (1999): after an accepted step
     * lambda *= max(1/3, 1 - (2 rho - 1)^3), after a rejected one lambda *= nu,
     * nu *= 2, where rho = actual / predicted decrease of chi^2. */
    double H[2][2], g[2];
    double chi2 = profiled_eval(&d, th[0], th[1], &I0, H, g);
    int evals = 1;
    double lambda = o->lm_lambda0, nu = 2.0;
    int it, converged = 0;
    for (it = 1; it <= o->max_iter_fit; ++it) {
        /* Stop test on the undamped Gauss-Newton step, the estimate of the
         * distance to the minimum that MIGRAD also stops on: a damped step can
         * be small far from the minimum of a flat valley when lambda is large. */
        if (gn_step(H, g, th, o, re_max) <= o->tol_fit) { converged = 1; break; }
        double M[2][2] = { { H[0][0] * (1.0 + lambda), H[0][1] },
                           { H[1][0], H[1][1] * (1.0 + lambda) } };
        double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        if (!(det > 0.0) || !isfinite(det)) { res->status |= ORC_FIT_SINGULAR; break; }
        double dt[2] = { (-M[1][1] * g[0] + M[0][1] * g[1]) / det,
                         (M[1][0] * g[0] - M[0][0] * g[1]) / det };
        double q[2] = { th[0] + dt[0], th[1] + dt[1] };
        clamp_theta(q, o, re_max);
        double s[2] = { q[0] - th[0], q[1] - th[1] };
        double Hq[2][2], gq[2], I0q;
        double chi2q = profiled_eval(&d, q[0], q[1], &I0q, Hq, gq);
        ++evals;
        /* predicted decrease of the Gauss-Newton model chi^2 + 2 g.s + s.H.s */
        double pred = -(2.0 * (g[0] * s[0] + g[1] * s[1])
                        + s[0] * (H[0][0] * s[0] + H[0][1] * s[1])
                        + s[1] * (H[1][0] * s[0] + H[1][1] * s[1]));
        if (chi2q < chi2) {
            double rho = pred > 0.0 ? (chi2 - chi2q) / pred : 1.0;
            double t = 2.0 * rho - 1.0;
            lambda *= fmax(1.0 / 3.0, 1.0 - t * t * t);
            nu = 2.0;
            th[0] = q[0]; th[1] = q[1];
            memcpy(H, Hq, sizeof H);
            memcpy(g, gq, sizeof g);
            chi2 = chi2q;
            I0 = I0q;
        } else {
            lambda *= nu;
            nu *= 2.0;
            if (lambda > 1e15) { converged = 1; break; }
        }
    }
    if (converged) res->status |= ORC_FIT_CONVERGED;
    else if (it > o->max_iter_fit) res->status |= ORC_FIT_MAXITER;
    if (th[0] <= o->re_min || th[0] >= re_max || th[1] <= o->n_min || th[1] >= o->n_max)
        res->status |= ORC_FIT_BOUND;
    if (!(I0 > 0.0)) res->status |= ORC_NONPOS_FLUX;
    res->I0 = I0;
    res->re = th[0];
    res->n = th[1];
    res->chi2 = chi2;
    res->it_fit = evals;   /* profile evaluations after the start */
    res->flux = orc_sersic_flux(I0, th[0], th[1], gabs);
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Public entry points (single stamp; pixels as float64, row-major).          */
/* ------------------------------------------------------------------------ */
/* The library's input contract: sides of 1 to 128 pixels (so h*w <= 128*128). */
static int size_ok(int h, int w) { return h >= 1 && w >= 1 && h <= 128 && w <= 128; }

/* Sec. 2 alone: brightest-pixel start, circular weight, centroid fixed point. */
void orc_centroid(const double *I, int h, int w, const orc_opts *o, orc_result *res)
{
    memset(res, 0, sizeof *res);
    res->npix = h * w;
    if (!size_ok(h, w)) { res->status |= ORC_BAD_SIZE; return; }
    int pr, pc;
    double r50;
    if (!init_stamp(I, h, w, &pr, &pc, &r50, &res->status)) return;
    double sw = clamp_sigw(r50 / SQRT_2LN2, h, w, &res->status);
    double xc = pc, yc = pr, g1 = 0.0, g2 = 0.0;
    moment_iterate(I, h, w, o, 0, &xc, &yc, &g1, &g2, &sw, &res->it_mom, &res->status);
    res->x0 = xc; res->y0 = yc; res->sigma_w = sw; res->r50 = r50;
}

/* Secs. 2-3 together from a given centre and sigma_w (g_w starts at 0, so the
 * first step is the circular-weight KSB estimate, Sec. 4.1). */
void orc_ellipticity(const double *I, int h, int w, const orc_opts *o, orc_result *res)
{
    uint32_t keep = res->status & (ORC_SIGW_CLAMPED | ORC_INIT_FALLBACK);
    res->status = keep;
    res->npix = h * w;
    if (!size_ok(h, w)) { res->status |= ORC_BAD_SIZE; return; }
    for (int p = 0; p < h * w; ++p) if (!isfinite(I[p])) { res->status |= ORC_NONFINITE; return; }
    double xc = res->x0, yc = res->y0, g1 = 0.0, g2 = 0.0, sw = res->sigma_w;
    moment_iterate(I, h, w, o, 1, &xc, &yc, &g1, &g2, &sw, &res->it_mom, &res->status);
    res->x0 = xc; res->y0 = yc; res->e1 = g1; res->e2 = g2; res->sigma_w = sw;
}

/* Sec. 4.1 profile fit with centre and ellipticity held fixed. */
void orc_sersic_fit(const double *I, const double *ivar, int h, int w, const orc_opts *o,
                    orc_result *res)
{
    res->npix = h * w;
    if (!size_ok(h, w)) { res->status |= ORC_BAD_SIZE; return; }
    fit_stamp(I, ivar, h, w, o, res->x0, res->y0, res->e1, res->e2, res->sigma_w, res, NULL);
}

/* The Sec. 4.1 fit with centre and ellipticity held fixed, started from a given
 * (r_e, n) instead of the Sec. 4.1 start (the candidates of n are still
 * evaluated, but not used).  For tests that check whether a lower chi^2 is a
 * different local minimum of the r_e - n valley. */
void orc_sersic_fit_from(const double *I, const double *ivar, int h, int w, const orc_opts *o,
                         double re0, double n0, orc_result *res)
{
    res->npix = h * w;
    if (!size_ok(h, w)) { res->status |= ORC_BAD_SIZE; return; }
    double start[2] = { re0, n0 };
    fit_stamp(I, ivar, h, w, o, res->x0, res->y0, res->e1, res->e2, res->sigma_w, res, start);
}

/* The whole chain of Sec. 4.1: start-up, centroid + ellipticity, fit. */
void orc_measure(const double *I, const double *ivar, int h, int w, const orc_opts *o,
                 orc_result *res)
{
    memset(res, 0, sizeof *res);
    res->npix = h * w;
    if (!size_ok(h, w)) { res->status |= ORC_BAD_SIZE; return; }
    int pr, pc;
    double r50;
    if (!init_stamp(I, h, w, &pr, &pc, &r50, &res->status)) return;
    double sw = clamp_sigw(r50 / SQRT_2LN2, h, w, &res->status);
    double xc = pc, yc = pr, g1 = 0.0, g2 = 0.0;
    moment_iterate(I, h, w, o, 1, &xc, &yc, &g1, &g2, &sw, &res->it_mom, &res->status);
    res->x0 = xc; res->y0 = yc; res->e1 = g1; res->e2 = g2; res->sigma_w = sw; res->r50 = r50;
    if (!(res->status & ORC_MOM_CONVERGED)) return;
    fit_stamp(I, ivar, h, w, o, xc, yc, g1, g2, sw, res, NULL);
}

/* One weighted pass exposed for the pins: e^obs, the centroid step and the
 * ellipticity step at a given (xc, yc, g_w, sigma_w). out = {dx, dy, dg1, dg2,
 * e1, e2, sigw_new, ok}. */
void orc_moment_step(const double *I, int h, int w, double xc, double yc, double g1,
                     double g2, double sw, double k_gain, int ellip, double out[8])
{
    moment_step s = weighted_pass(I, h, w, xc, yc, g1, g2, sw, k_gain, ellip);
    out[0] = s.dx; out[1] = s.dy; out[2] = s.dg1; out[3] = s.dg2;
    out[4] = s.e1; out[5] = s.e2; out[6] = s.sigw_new; out[7] = s.ok;
}

/* chi^2 and normal equations at given (I0, r_e, n) with the centre and
 * ellipticity fixed; out = {chi2, g[3], H[9]}. */
void orc_fit_eval_ss(const double *I, const double *ivar, int h, int w, double xc, double yc,
                     double g1, double g2, const double p[3], int supersample, double out[13])
{
    int npix = h * w;
    int S = supersample > 1 ? supersample : 1;
    double *r = sample_radii(h, w, S, xc, yc, g1, g2);
    fit_data d = { I, ivar, r, npix, S * S };
    double H[3][3], g[3];
    out[0] = fit_eval(&d, p, H, g);
    for (int a = 0; a < 3; ++a) out[1 + a] = g[a];
    for (int a = 0; a < 3; ++a) for (int c = 0; c < 3; ++c) out[4 + 3 * a + c] = H[a][c];
    free(r);
}

void orc_fit_eval(const double *I, const double *ivar, int h, int w, double xc, double yc,
                  double g1, double g2, const double p[3], double out[13])
{
    orc_fit_eval_ss(I, ivar, h, w, xc, yc, g1, g2, p, 1, out);
}

/* Gradient of chi^2 (Eq. 11) for the elliptical Sérsic model of Eq. 10 with
 * respect to all seven parameters p = (x0, y0, g1, g2, I0, r_e, n) and to the
 * pixels.  With r_i = m_i - I_i and weights w_i (1/sigma_i^2, default 1):
 *   chi^2 = sum w r^2,   dchi^2/dp = 2 sum w r dm/dp,   dchi^2/dI_i = -2 w_i r_i.
 * The model depends on the centre and the ellipticity only through the
 * Sérsic radius r = sqrt(R^2(theta; g)) / (1 - |g|) (R^2 from Eq. A1), so
 *   dm/dq = dm/dr * dr/dq,   dm/dr = -m b u / (n r),   u = (r / r_e)^(1/n),
 *   dr/dR^2 = r / (2 R^2),   dr/d|g| = r / (1 - |g|),   d|g|/dg_k = g_k / |g|.
 * The pixel at R^2 = 0 adds no centre or shape derivative (the profile has a
 * cusp there for n > 1), and d|g|/dg is taken as 0 at g = 0 (the kink).
 * Writes chi^2, grad[7] and, if dpix != NULL, the h*w pixel gradient.
 * If scale != NULL it also writes the first-order error scales of a
 * lower-precision evaluation: scale[k] = sum_i 2 w_i |dm_i/dp_k| (|m_i| + |r_i|)
 * for k < 7 and scale[7] = sum_i 2 w_i |r_i| (|m_i| + |r_i|).  An
 * implementation whose per-pixel m and r carry relative errors up to eps
 * differs from grad[k] and chi^2 by at most about eps * scale[k]. */
void orc_chi2_grad(const double *I, const double *ivar, int h, int w, const double p[7],
                   double *chi2_out, double grad[7], double *dpix, double scale[8])
{
    const double x0 = p[0], y0 = p[1], g1 = p[2], g2 = p[3], I0 = p[4], re = p[5], n = p[6];
    const double gabs = sqrt(g1 * g1 + g2 * g2);
    const double b = orc_sersic_b(n), db = orc_sersic_db(n);
    /* R^2 = A t1^2 + B t2^2 - 4 g2 t1 t2 and the derivatives of its coefficients */
    const double A = (1.0 - g1) * (1.0 - g1) + g2 * g2;
    const double B = (1.0 + g1) * (1.0 + g1) + g2 * g2;
    const double dA_g1 = -2.0 * (1.0 - g1), dB_g1 = 2.0 * (1.0 + g1);
    const double dA_g2 = 2.0 * g2, dB_g2 = 2.0 * g2;
    const double dabs1 = gabs > 0.0 ? g1 / gabs : 0.0, dabs2 = gabs > 0.0 ? g2 / gabs : 0.0;
    double chi2 = 0.0;
    for (int a = 0; a < 7; ++a) grad[a] = 0.0;
    if (scale) for (int a = 0; a < 8; ++a) scale[a] = 0.0;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            const int k = i * w + j;
            double dm[7] = { 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0 };   /* dm/dp, for scale */
            const double t1 = j - x0, t2 = i - y0;
            const double R2 = ellip_R2(t1, t2, g1, g2);
            const double r = sqrt(R2 > 0.0 ? R2 : 0.0) / (1.0 - gabs);
            const double x = r / re;
            const double u = x > 0.0 ? pow(x, 1.0 / n) : 0.0;
            const double E = exp(-b * u);
            const double m = I0 * E;
            const double wgt = ivar ? ivar[k] : 1.0;
            const double res = m - I[k];
            const double c = 2.0 * wgt * res;
            chi2 += wgt * res * res;
            dm[4] = E;                                               /* dm/dI0 */
            dm[5] = m * b * u / (n * re);                            /* dm/dr_e */
            if (x > 0.0) dm[6] = m * u * (b * log(x) / (n * n) - db);   /* dm/dn */
            if (R2 > 0.0) {
                const double dm_dr = -m * b * u / (n * r);
                const double dr_dR2 = r / (2.0 * R2);
                const double dR2_x0 = -(2.0 * A * t1 - 4.0 * g2 * t2);
                const double dR2_y0 = -(2.0 * B * t2 - 4.0 * g2 * t1);
                const double dR2_g1 = dA_g1 * t1 * t1 + dB_g1 * t2 * t2;
                const double dR2_g2 = dA_g2 * t1 * t1 + dB_g2 * t2 * t2 - 4.0 * t1 * t2;
                const double dr_g1 = dr_dR2 * dR2_g1 + r / (1.0 - gabs) * dabs1;
                const double dr_g2 = dr_dR2 * dR2_g2 + r / (1.0 - gabs) * dabs2;
                dm[0] = dm_dr * dr_dR2 * dR2_x0;
                dm[1] = dm_dr * dr_dR2 * dR2_y0;
                dm[2] = dm_dr * dr_g1;
                dm[3] = dm_dr * dr_g2;
            }
            for (int a = 0; a < 7; ++a) grad[a] += c * dm[a];
            if (scale) {
                const double mag = 2.0 * wgt * (fabs(m) + fabs(res));
                for (int a = 0; a < 7; ++a) scale[a] += mag * fabs(dm[a]);
                scale[7] += mag * fabs(res);
            }
            if (dpix) dpix[k] = -c;
        }
    *chi2_out = chi2;
}

/* ------------------------------------------------------------------------ */
/* Star profiles (Sec. 4.2): size and amplitude from weighted radial moments */
/* ------------------------------------------------------------------------ */
/* The radial moments r_k = sum I W r^k over the pixels, with the centre and
 * the ellipticity held fixed and r the semi-major-axis radius of Eq. A1,
 * r = R(g) / (1 - |g|) (the paper writes the circular case; for an elliptical
 * profile the pixel sums carry the axis ratio q = (1-|g|)/(1+|g|) as the
 * Jacobian of the elliptical coordinates, which cancels from every ratio).
 *   Gaussian (Eqs. gau...): W = exp(-r^2 / 2 s_w^2).  With s_w = s,
 *     r0 = pi s^2 I0 q,  r2 = pi s^4 I0 q,  so s = sqrt(r2 / r0),
 *     I0 = r0 / (pi s^2 q); s_w <- s is iterated to its fixed point.
 *   Moffat: W = (1 + r^2 / r_dw^2)^-3.  With r_dw = r_d,
 *     r0 = I0 q pi r_d^2 / (b+2),  r2 = I0 q pi r_d^4 / ((b+1)(b+2)),
 *     r4 = I0 q 2 pi r_d^6 / (b (b+1)(b+2)),
 *   so b = 1 / (r4 r0 / (2 r2^2) - 1), r_d = sqrt(r2 / r0 (b+1)),
 *   I0 = r0 (b+2) / (pi r_d^2 q); r_dw <- r_d is iterated.
 * Also: flux (Gaussian 2 pi s^2 I0 q, Moffat pi r_d^2 I0 q / (b-1)) and the
 * half-light radius along the major axis (Gaussian s sqrt(2 ln 2), Moffat
 * r_d sqrt(2^(1/(b-1)) - 1)). */
typedef struct {
    double size, beta, I0, flux, r50;
    int32_t iters;
    uint32_t status;
} orc_star_result;

static void star_moments(const double *I, int h, int w, double xc, double yc, double g1, double g2,
                         int profile, double size_w, double m[3])
{
    double gabs = sqrt(g1 * g1 + g2 * g2);
    m[0] = m[1] = m[2] = 0.0;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            double R2 = ellip_R2(j - xc, i - yc, g1, g2);
            double r2 = (R2 > 0.0 ? R2 : 0.0) / ((1.0 - gabs) * (1.0 - gabs));
            double W;
            if (profile == 0) {
                W = exp(-r2 / (2.0 * size_w * size_w));
            } else {
                double t = 1.0 + r2 / (size_w * size_w);
                W = 1.0 / (t * t * t);
            }
            double f = I[i * w + j] * W;
            m[0] += f;
            m[1] += f * r2;
            m[2] += f * r2 * r2;
        }
}

/* profile 0 = Gaussian, 1 = Moffat; size0 > 0 starts the weight size. */
void orc_star(const double *I, int h, int w, const orc_opts *o, int profile, double xc, double yc,
              double g1, double g2, double size0, orc_star_result *res)
{
    memset(res, 0, sizeof *res);
    if (h < 1 || w < 1 || (int64_t)h * w > 128 * 128) { res->status |= ORC_BAD_SIZE; return; }
    for (int p = 0; p < h * w; ++p) if (!isfinite(I[p])) { res->status |= ORC_NONFINITE; return; }
    double gabs = sqrt(g1 * g1 + g2 * g2);
    double q = (1.0 - gabs) / (1.0 + gabs);
    double sw = size0, size = size0, beta = 0.0, m[3];
    int it;
    for (it = 1; it <= o->max_iter_mom; ++it) {
        star_moments(I, h, w, xc, yc, g1, g2, profile, sw, m);
        if (!(m[0] > 0.0) || !(m[1] > 0.0)) { res->status |= ORC_MOM_FAILED; break; }
        if (profile == 0) {
            size = sqrt(m[1] / m[0]);
        } else {
            double ratio = m[2] * m[0] / (2.0 * m[1] * m[1]);
            if (!(ratio > 1.0)) { res->status |= ORC_MOM_FAILED; break; }
            beta = 1.0 / (ratio - 1.0);
            size = sqrt(m[1] / m[0] * (beta + 1.0));
        }
        if (!isfinite(size) || !(size > 0.0)) { res->status |= ORC_MOM_FAILED; break; }
        double step = fabs(size / sw - 1.0);
        sw = size;
        if (step <= o->tol_sig) { res->status |= ORC_MOM_CONVERGED; break; }
    }
    if (it > o->max_iter_mom) { res->status |= ORC_MOM_MAXITER; it = o->max_iter_mom; }
    res->iters = it;
    res->size = size;
    res->beta = beta;
    if (!(res->status & ORC_MOM_CONVERGED)) return;
    /* the closed forms at the fixed point, from the moments of the last pass */
    if (profile == 0) {
        res->I0 = m[0] / (M_PI * size * size * q);
        res->flux = 2.0 * M_PI * size * size * res->I0 * q;
        res->r50 = size * SQRT_2LN2;
    } else {
        res->I0 = m[0] * (beta + 2.0) / (M_PI * size * size * q);
        res->flux = beta > 1.0 ? M_PI * size * size * res->I0 * q / (beta - 1.0) : INFINITY;
        res->r50 = beta > 1.0 ? size * sqrt(pow(2.0, 1.0 / (beta - 1.0)) - 1.0) : INFINITY;
    }
}

/* ------------------------------------------------------------------------ */
/* Implicit gradients of the moment fixed point (Secs. 2-3).                  */
/* ------------------------------------------------------------------------ */
/* The moment iteration stops where its steps vanish.  With
 * theta = (xc, yc, g1, g2, sigma_w), t = pixel - centre, R^2 of Eq. A1 at g,
 * W = exp(-R^2 / 2 sigma_w^2) and e_w = 2 g / (1 + g^2), that point solves
 *   F1 = sum I W t1 = 0,  F2 = sum I W t2 = 0          zero centroid step (Eqs. 3-6)
 *   F3 = sum I W [(t1^2 - t2^2) - e_w1 (t1^2 + t2^2)]   e^obs = e_w, the zero of
 *   F4 = sum I W [2 t1 t2 - e_w2 (t1^2 + t2^2)]           the step of Eq. 9, times T
 *   F5 = sum I W [R^2 - sigma_w^2] = 0                  the matched weight,
 *                                                       sigma_w^2 = sum I W R^2 / sum I W
 * Each F_k = sum_p I_p psi_k(p; theta) is linear in the pixels, so by the
 * implicit function theorem d theta / d I_p = -J^-1 psi(p; theta), with
 * J_kl = sum_p I_p d psi_k / d theta_l.
 * mode bit 0 (ORC_MOM_ELLIP): g is a parameter (the Secs. 2-3 fixed point);
 * without it g = 0 is held (Sec. 2 alone: F3, F4 dropped).  sigma_w follows
 * one of three rules:
 *   (default)            the matched weight, F5 above;
 *   ORC_MOM_SIGW_FIXED   held (F5 dropped; d sigma_w = 0), e.g. a clamped weight;
 *   ORC_MOM_SIGW_R50     sigma_w = r50 / sqrt(2 ln 2) with r50 from the growth
 *                        curve of the start-up (Sec. 4.1): F5 is dropped and
 *                        sigma_w enters as an explicit function of the pixels,
 *                        d theta_a = -J_aa^-1 (psi_a + J_as d sigma_w).
 * Held parameters have zero derivatives. */
#define ORC_MOM_ELLIP      1
#define ORC_MOM_SIGW_FIXED 2
#define ORC_MOM_SIGW_R50   4

/* d sigma_w / d I_p for sigma_w = r50 / sqrt(2 ln 2).  r50 interpolates
 * linearly in the ring k that crosses half the total H:
 *   r50 = (k - 1) + (H - P) / (S - P),  P, S = sums over the discs d <= k-1, d <= k
 *   (k = 0: r50 = H / (2 S), S the brightest pixel),
 * with the brightest pixel and k held (they change only at isolated points).
 * The derivative is zero where r50 is the fallback or sigma_w is clamped.
 * Returns 1 if sigma_w depends on the pixels. */
static int sigw_r50_grad(const double *I, int h, int w, double *ds)
{
    int pr, pc, k;
    double r50;
    uint32_t st = 0;
    for (int p = 0; p < h * w; ++p) ds[p] = 0.0;
    if (!init_stamp_k(I, h, w, &pr, &pc, &r50, &st, &k) || k < 0) return 0;
    uint32_t cl = 0;
    clamp_sigw(r50 / SQRT_2LN2, h, w, &cl);
    if (cl) return 0;
    double H = 0.0, P = 0.0, S = 0.0;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            int d2 = (i - pr) * (i - pr) + (j - pc) * (j - pc);
            H += 0.5 * I[i * w + j];
            if (k >= 1 && d2 <= (k - 1) * (k - 1)) P += I[i * w + j];
            if (d2 <= k * k) S += I[i * w + j];
        }
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            int d2 = (i - pr) * (i - pr) + (j - pc) * (j - pc);
            double inP = (k >= 1 && d2 <= (k - 1) * (k - 1)) ? 1.0 : 0.0;
            double inS = d2 <= k * k ? 1.0 : 0.0;
            double dr;
            if (k == 0) dr = 0.5 * (0.5 * S - H * inS) / (S * S);
            else dr = ((0.5 - inP) * (S - P) - (H - P) * (inS - inP)) / ((S - P) * (S - P));
            ds[i * w + j] = dr / SQRT_2LN2;
        }
    return 1;
}

static int moment_is_active(int mode, int l)
{
    if ((l == 2 || l == 3) && !(mode & ORC_MOM_ELLIP)) return 0;
    if (l == 4 && (mode & (ORC_MOM_SIGW_FIXED | ORC_MOM_SIGW_R50))) return 0;
    return 1;
}

/* psi_k(p; theta) and, if dpsi != NULL, d psi_k / d theta_l (row k, column l). */
static void moment_psi(double t1, double t2, const double th[5], double psi[5], double dpsi[5][5])
{
    double g1 = th[2], g2 = th[3], s = th[4];
    double gg = g1 * g1 + g2 * g2;
    double A = 1.0 + gg - 2.0 * g1, B = 1.0 + gg + 2.0 * g1;
    double R2 = ellip_R2(t1, t2, g1, g2);
    double W = exp(-R2 / (2.0 * s * s));
    double ew1 = 2.0 * g1 / (1.0 + gg), ew2 = 2.0 * g2 / (1.0 + gg);
    double th2 = t1 * t1 + t2 * t2;
    double m[5] = { t1, t2, (t1 * t1 - t2 * t2) - ew1 * th2, 2.0 * t1 * t2 - ew2 * th2, R2 - s * s };
    for (int k = 0; k < 5; ++k) psi[k] = W * m[k];
    if (!dpsi) return;
    /* derivatives of R^2 (t1 = x - xc, t2 = y - yc, so d t / d xc = -1) */
    double dR2[5];
    dR2[0] = -(2.0 * A * t1 - 4.0 * g2 * t2);
    dR2[1] = -(2.0 * B * t2 - 4.0 * g2 * t1);
    dR2[2] = (2.0 * g1 - 2.0) * t1 * t1 + (2.0 * g1 + 2.0) * t2 * t2;
    dR2[3] = 2.0 * g2 * th2 - 4.0 * t1 * t2;
    dR2[4] = 0.0;
    /* derivatives of W: through R^2, and through sigma_w */
    double dW[5];
    for (int l = 0; l < 4; ++l) dW[l] = -W * dR2[l] / (2.0 * s * s);
    dW[4] = W * R2 / (s * s * s);
    /* derivatives of e_w = 2 g / (1 + g^2) */
    double q = (1.0 + gg) * (1.0 + gg);
    double dew1[2] = { 2.0 * (1.0 - g1 * g1 + g2 * g2) / q, -4.0 * g1 * g2 / q };
    double dew2[2] = { -4.0 * g1 * g2 / q, 2.0 * (1.0 + g1 * g1 - g2 * g2) / q };
    /* derivatives of the polynomial factors m_k */
    double dm[5][5] = { { 0 } };
    dm[0][0] = -1.0;
    dm[1][1] = -1.0;
    dm[2][0] = -2.0 * t1 + ew1 * 2.0 * t1;
    dm[2][1] = 2.0 * t2 + ew1 * 2.0 * t2;
    dm[2][2] = -dew1[0] * th2;
    dm[2][3] = -dew1[1] * th2;
    dm[3][0] = -2.0 * t2 + ew2 * 2.0 * t1;
    dm[3][1] = -2.0 * t1 + ew2 * 2.0 * t2;
    dm[3][2] = -dew2[0] * th2;
    dm[3][3] = -dew2[1] * th2;
    for (int l = 0; l < 4; ++l) dm[4][l] = dR2[l];
    dm[4][4] = -2.0 * s;
    for (int k = 0; k < 5; ++k)
        for (int l = 0; l < 5; ++l) dpsi[k][l] = dW[l] * m[k] + W * dm[k][l];
}

/* F(theta) and J = dF/dtheta over the whole stamp (all 5 x 5 entries). */
void orc_moment_jacobian(const double *I, int h, int w, const double th[5], double F[5], double J[25])
{
    double psi[5], dpsi[5][5];
    for (int k = 0; k < 5; ++k) F[k] = 0.0;
    for (int k = 0; k < 25; ++k) J[k] = 0.0;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            double f = I[i * w + j];
            moment_psi(j - th[0], i - th[1], th, psi, dpsi);
            for (int k = 0; k < 5; ++k) {
                F[k] += f * psi[k];
                for (int l = 0; l < 5; ++l) J[k * 5 + l] += f * dpsi[k][l];
            }
        }
}

/* Solve M x = b (n x n, row-major, n <= 5) by Gaussian elimination with
 * partial pivoting; returns 0, or 1 if M is singular. */
static int solve_small(int n, const double *M_in, const double *b_in, double *x)
{
    double M[25], b[5], big = 0.0;
    for (int k = 0; k < n * n; ++k) { M[k] = M_in[k]; if (fabs(M[k]) > big) big = fabs(M[k]); }
    for (int k = 0; k < n; ++k) b[k] = b_in[k];
    if (!(big > 0.0)) return 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (fabs(M[r * n + c]) > fabs(M[piv * n + c])) piv = r;
        if (!(fabs(M[piv * n + c]) > 1e-14 * big)) return 1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = M[r * n + c] / M[c * n + c];
            for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= M[r * n + k] * x[k];
        x[r] = acc / M[r * n + r];
    }
    return 0;
}

/* The active block of J (rows and columns of the active parameters), or its
 * transpose; returns the number of active parameters and their indices. */
static int moment_active_block(const double J[25], int mode, int transpose, double *Ja, int act[5])
{
    int n = 0;
    for (int l = 0; l < 5; ++l) if (moment_is_active(mode, l)) act[n++] = l;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            Ja[a * n + b] = transpose ? J[act[b] * 5 + act[a]] : J[act[a] * 5 + act[b]];
    return n;
}

/* JVP: the derivative of theta along a pixel tangent u,
 *   dtheta_a = -J_aa^-1 (sum_p u_p psi_a(p) + J_as dsigma_w),
 * dsigma_w = sum_p u_p d sigma_w / d I_p under ORC_MOM_SIGW_R50 (else 0).
 * Returns 0, or 1 if J_aa is singular (dtheta = 0). */
int orc_moment_jvp(const double *I, int h, int w, const double th[5], int mode, const double *u,
                   double dth[5])
{
    double F[5], J[25], Ja[25], rhs[5] = { 0 }, x[5], S[5] = { 0 }, psi[5], dsw = 0.0;
    int act[5];
    for (int l = 0; l < 5; ++l) dth[l] = 0.0;
    orc_moment_jacobian(I, h, w, th, F, J);
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            moment_psi(j - th[0], i - th[1], th, psi, NULL);
            for (int k = 0; k < 5; ++k) S[k] += u[i * w + j] * psi[k];
        }
    if (mode & ORC_MOM_SIGW_R50) {
        double *ds = (double *)malloc(sizeof(double) * h * w);
        if (sigw_r50_grad(I, h, w, ds))
            for (int p = 0; p < h * w; ++p) dsw += u[p] * ds[p];
        free(ds);
    }
    int n = moment_active_block(J, mode, 0, Ja, act);
    for (int a = 0; a < n; ++a) rhs[a] = -(S[act[a]] + J[act[a] * 5 + 4] * dsw);
    if (solve_small(n, Ja, rhs, x)) return 1;
    for (int a = 0; a < n; ++a) dth[act[a]] = x[a];
    if (mode & ORC_MOM_SIGW_R50) dth[4] = dsw;
    return 0;
}

/* VJP: dL/dI for v = dL/dtheta (entries of held parameters ignored):
 *   J_aa^T lambda = v_a,
 *   dL/dI_p = -lambda . psi_a(p) + (v_s - lambda . J_as) d sigma_w / d I_p
 * (the last term under ORC_MOM_SIGW_R50 only).  Returns 0, or 1 if J_aa is
 * singular (dI = 0). */
int orc_moment_vjp(const double *I, int h, int w, const double th[5], int mode, const double v[5],
                   double *dI)
{
    double F[5], J[25], Ja[25], rhs[5] = { 0 }, lam_a[5], lam[5] = { 0 }, psi[5];
    int act[5];
    for (int p = 0; p < h * w; ++p) dI[p] = 0.0;
    orc_moment_jacobian(I, h, w, th, F, J);
    int n = moment_active_block(J, mode, 1, Ja, act);
    for (int a = 0; a < n; ++a) rhs[a] = v[act[a]];
    if (solve_small(n, Ja, rhs, lam_a)) return 1;
    for (int a = 0; a < n; ++a) lam[act[a]] = lam_a[a];
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j) {
            moment_psi(j - th[0], i - th[1], th, psi, NULL);
            double acc = 0.0;
            for (int k = 0; k < 5; ++k) acc += lam[k] * psi[k];
            dI[i * w + j] = -acc;
        }
    if (mode & ORC_MOM_SIGW_R50) {
        double kappa = v[4];
        for (int k = 0; k < 5; ++k) kappa -= lam[k] * J[k * 5 + 4];
        double *ds = (double *)malloc(sizeof(double) * h * w);
        if (sigw_r50_grad(I, h, w, ds))
            for (int p = 0; p < h * w; ++p) dI[p] += kappa * ds[p];
        free(ds);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The cut-out of Sec. 4.1: a square of side six times r50 around the        */
/* brightest pixel of a large image.                                         */
/* ------------------------------------------------------------------------ */
/* r50 is the start-up growth curve around the brightest pixel (the same as
 * the stamp start-up).  The side is side_factor * r50 rounded to the nearest
 * integer (halves up), clamped to [min_side, max_side]; the square starts
 * side/2 (integer division) rows and columns before the brightest pixel and is
 * cut to the image.  NONFINITE: no cut-out (h = w = 0). */
typedef struct {
    int32_t row0, col0, h, w;
    double r50;
    uint32_t status;
} orc_cutout_info;

void orc_cutout(const double *I, int H, int W, double side_factor, int min_side, int max_side,
                orc_cutout_info *out)
{
    int pr, pc;
    double r50;
    uint32_t st = 0;
    memset(out, 0, sizeof *out);
    if (!init_stamp(I, H, W, &pr, &pc, &r50, &st)) { out->status = st; return; }
    long side = (long)floor(side_factor * r50 + 0.5);
    if (side < min_side) side = min_side;
    if (side > max_side) side = max_side;
    int r0 = pr - (int)(side / 2), c0 = pc - (int)(side / 2);
    int r1 = r0 + (int)side, c1 = c0 + (int)side;
    if (r0 < 0) r0 = 0;
    if (c0 < 0) c0 = 0;
    if (r1 > H) r1 = H;
    if (c1 > W) c1 = W;
    out->row0 = r0;
    out->col0 = c0;
    out->h = r1 - r0;
    out->w = c1 - c0;
    out->r50 = r50;
    out->status = st;
}

/* Batch over a flat fp32 buffer (stamp s at pix + offset[s], h[s] x w[s]),
 * parallel over stamps with OpenMP.  stage: 0 = whole chain (orc_measure),
 * 1 = centroid, 2 = ellipticity (uses res[s] x0, y0, sigma_w), 3 = fit (uses
 * res[s] x0, y0, e1, e2, sigma_w).  Returns the number of threads used. */
int orc_batch(const float *pix, const int64_t *offset, const int32_t *h, const int32_t *w,
              int64_t count, const float *ivar, const orc_opts *o, int stage,
              orc_result *res, int threads)
{
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < count; ++s) {
        int hh = h[s], ww = w[s];
        if (!size_ok(hh, ww)) {
            memset(&res[s], 0, sizeof res[s]);
            res[s].status = ORC_BAD_SIZE;
            continue;
        }
        int np = hh * ww;
        double *I = (double *)malloc(sizeof(double) * np);
        double *iv = ivar ? (double *)malloc(sizeof(double) * np) : NULL;
        for (int p = 0; p < np; ++p) I[p] = pix[offset[s] + p];
        if (iv) for (int p = 0; p < np; ++p) iv[p] = ivar[offset[s] + p];
        switch (stage) {
        case 0: orc_measure(I, iv, hh, ww, o, &res[s]); break;
        case 1: orc_centroid(I, hh, ww, o, &res[s]); break;
        case 2: orc_ellipticity(I, hh, ww, o, &res[s]); break;
        default: orc_sersic_fit(I, iv, hh, ww, o, &res[s]); break;
        }
        free(I);
        free(iv);
    }
    return used;
}
