// fse_moment_grad.cu -- implicit-function derivatives of the moment fixed
// point (Secs. 2-3) with respect to the pixels: VJP (fse_moment_vjp) and JVP
// (fse_moment_jvp).
//
// The moment iteration stops where its steps vanish.  With theta = (xc, yc,
// g1, g2, sigma_w), t = pixel - centre, R^2 of Eq. A1, W = exp(-R^2/2 s^2) and
// e_w = 2g/(1+g^2), that point solves F_k = sum_p I_p W m_k(t) = 0 with
//   m_1 = t1, m_2 = t2                         zero centroid step (Eqs. 3-6)
//   m_3 = (t1^2 - t2^2) - e_w1 (t1^2 + t2^2)   e^obs = e_w, where the step of
//   m_4 = 2 t1 t2 - e_w2 (t1^2 + t2^2)         Eq. 9 vanishes
//   m_5 = R^2 - s^2                            matched weight
// so d theta / d I_p = -J^-1 W(p) m(p) with J_kl = sum_p I_p d(W m_k)/d theta_l.
// Every m_k and every d R^2 / d theta_l is a polynomial of degree <= 2 in t,
// so J is a fixed combination of the 15 weighted moments
// M_ab = sum I W t1^a t2^b (a + b <= 4): one pass accumulates them, 25 lanes
// assemble one entry of J each, and every lane solves the 5 x 5 system.
// sigma_w from the start-up growth curve (r50 / sqrt(2 ln 2), Sec. 4.1) is
// an explicit function of the pixels: it is piecewise constant in the three
// regions of the crossing ring (inside the disc k-1, in ring k, outside),
// found from double-float disc sums around the brightest pixel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fse_device.cuh"
#include "fse_internal.h"

namespace fse {
namespace {

constexpr float kInvSqrt2Ln2F = 0.849321800f;   // 1 / sqrt(2 ln 2)

// Index of the monomial t1^a t2^b among the 15 of degree <= 4, by degree and
// then by the power of t2.
__host__ __device__ constexpr int mono(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }
// The six monomials of degree <= 2: 1, t1, t2, t1^2, t1 t2, t2^2.
__host__ __device__ constexpr int pa(int i) { return i == 1 || i == 3 || i == 4 ? (i == 3 ? 2 : 1) : 0; }
__host__ __device__ constexpr int pb(int i) { return i == 2 || i == 4 || i == 5 ? (i == 5 ? 2 : 1) : 0; }

template <int DT>
__device__ __forceinline__ float load_pix(const MomentGradArgs& a, int64_t off, float sc) {
    return DT == FSE_BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.pix)[off]) * sc
                          : __ldg(static_cast<const float*>(a.pix) + off);
}

// Stamp geometry at theta.
struct Geom {
    float x0, y0, g1, g2, s;
    float A, B, G4, cw;      // R^2 = A t1^2 + B t2^2 - G4 t1 t2; W = 2^(cw R^2)
};

// Polynomial factors of degree <= 2 (coefficients of 1, t1, t2, t1^2, t1 t2,
// t2^2) for J_kl = sum I W [a_l m_k + dm_k/dtheta_l]: m_k, a_l (the derivative
// of log W: -R^2_l / 2 s^2, or R^2 / s^3 for sigma_w) and dm_k/dtheta_l.
__device__ void jac_polys(const Geom& q, int k, int l, float mk[6], float al[6], float dm[6]) {
    const float g1 = q.g1, g2 = q.g2, s = q.s, gg = g1 * g1 + g2 * g2;
    const float ew1 = 2.f * g1 / (1.f + gg), ew2 = 2.f * g2 / (1.f + gg);
    const float qq = (1.f + gg) * (1.f + gg);
    const float dew[2][2] = {{2.f * (1.f - g1 * g1 + g2 * g2) / qq, -4.f * g1 * g2 / qq},
                             {-4.f * g1 * g2 / qq, 2.f * (1.f + g1 * g1 - g2 * g2) / qq}};
#pragma unroll
    for (int i = 0; i < 6; ++i) mk[i] = al[i] = dm[i] = 0.f;
    // d R^2 / d theta_l
    float du[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (l == 0) { du[1] = -2.f * q.A; du[2] = q.G4; }
    if (l == 1) { du[1] = q.G4; du[2] = -2.f * q.B; }
    if (l == 2) { du[3] = 2.f * (g1 - 1.f); du[5] = 2.f * (g1 + 1.f); }
    if (l == 3) { du[3] = 2.f * g2; du[4] = -4.f; du[5] = 2.f * g2; }
    const float c = 1.f / (2.f * s * s);
    if (l < 4) {
#pragma unroll
        for (int i = 0; i < 6; ++i) al[i] = -c * du[i];
    } else {
        const float is3 = 1.f / (s * s * s);
        al[3] = q.A * is3; al[4] = -q.G4 * is3; al[5] = q.B * is3;
    }
    if (k == 0) { mk[1] = 1.f; if (l == 0) dm[0] = -1.f; }
    if (k == 1) { mk[2] = 1.f; if (l == 1) dm[0] = -1.f; }
    if (k == 2) {
        mk[3] = 1.f - ew1; mk[5] = -(1.f + ew1);
        if (l == 0) dm[1] = -2.f * (1.f - ew1);
        if (l == 1) dm[2] = 2.f * (1.f + ew1);
        if (l == 2 || l == 3) { dm[3] = dm[5] = -dew[0][l - 2]; }
    }
    if (k == 3) {
        mk[3] = -ew2; mk[4] = 2.f; mk[5] = -ew2;
        if (l == 0) { dm[1] = 2.f * ew2; dm[2] = -2.f; }
        if (l == 1) { dm[1] = -2.f; dm[2] = 2.f * ew2; }
        if (l == 2 || l == 3) { dm[3] = dm[5] = -dew[1][l - 2]; }
    }
    if (k == 4) {
        mk[0] = -s * s; mk[3] = q.A; mk[4] = -q.G4; mk[5] = q.B;
        if (l < 4) {
#pragma unroll
            for (int i = 0; i < 6; ++i) dm[i] = du[i];
        } else {
            dm[0] = -2.f * s;
        }
    }
}

// Double-float helpers: the exact product error by FMA, Knuth's two-sum.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void df_acc(float& hi, float& lo, float p, float e) {
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
}

// One entry of J from the 15 moments (hi + lo pairs).  The combination
// cancels by up to an order of magnitude (e.g. J_55 = sum I W [R^2 (R^2 - s^2)
// / s^3 - 2 s]), so each coefficient, product and partial sum is carried in
// double-float: once per stamp, 42 terms per lane.
__device__ float jac_entry(const Geom& q, int k, int l, const float Mh[15], const float Ml[15]) {
    float mk[6], al[6], dm[6];
    jac_polys(q, k, l, mk, al, dm);
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int a = mono(pa(i), pb(i));
        float p, e;
        two_prod(dm[i], Mh[a], p, e);
        df_acc(hi, lo, p, fmaf(dm[i], Ml[a], e));
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const int b = mono(pa(i) + pa(j), pb(i) + pb(j));
            float ch, cl;
            two_prod(al[i], mk[j], ch, cl);
            two_prod(ch, Mh[b], p, e);
            df_acc(hi, lo, p, fmaf(ch, Ml[b], fmaf(cl, Mh[b], e)));
        }
    }
    return hi + lo;
}

// Solve X x = r for 5 x 5 X (row-major) by Gaussian elimination with partial
// pivoting, every index known at compile time.  Returns false if a pivot is
// below 1e-6 of the largest entry.
__device__ bool solve5(float X[25], float r[5], float x[5]) {
    float big = 0.f;
#pragma unroll
    for (int i = 0; i < 25; ++i) big = fmaxf(big, fabsf(X[i]));
    if (!(big > 0.f)) return false;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        float pv = fabsf(X[c * 5 + c]);
#pragma unroll
        for (int rr = c + 1; rr < 5; ++rr)
            if (fabsf(X[rr * 5 + c]) > pv) { pv = fabsf(X[rr * 5 + c]); piv = rr; }
        if (!(pv > 1e-6f * big)) return false;
#pragma unroll
        for (int rr = c + 1; rr < 5; ++rr) {
            if (rr == piv) {
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float t = X[c * 5 + k];
                    X[c * 5 + k] = X[rr * 5 + k];
                    X[rr * 5 + k] = t;
                }
                const float t = r[c];
                r[c] = r[rr];
                r[rr] = t;
            }
        }
        const float inv = 1.f / X[c * 5 + c];
#pragma unroll
        for (int rr = c + 1; rr < 5; ++rr) {
            const float f = X[rr * 5 + c] * inv;
#pragma unroll
            for (int k = c; k < 5; ++k) X[rr * 5 + k] = fmaf(-f, X[c * 5 + k], X[rr * 5 + k]);
            r[rr] = fmaf(-f, r[c], r[rr]);
        }
    }
#pragma unroll
    for (int rr = 4; rr >= 0; --rr) {
        float acc = r[rr];
#pragma unroll
        for (int k = rr + 1; k < 5; ++k) acc = fmaf(-X[rr * 5 + k], x[k], acc);
        x[rr] = acc / X[rr * 5 + rr];
    }
    return true;
}

// The growth curve of the start-up (Sec. 4.1) around the brightest pixel:
// the crossing ring k (the first whose enclosed sum reaches half the total)
// and the constants of d sigma_w / d I_p in the three regions d <= k-1,
// k-1 < d <= k and d > k.  The disc sums are double-float, so k is the
// start-up's own except where an enclosed sum lies within ~1e-13 of half the
// total.  For the JVP the tangent's sums over the two discs come with them.

template <int DT, bool JVP>
__device__ R50Grad r50_ring(const MomentGradArgs& a, const fse_stamp& ix, int npix, float sc, float r50_hint,
                            int peak, float tot_h, float tot_l, int lane) {
    R50Grad o;
    o.on = 0;
    o.pr = peak / ix.w;
    o.pc = peak - o.pr * ix.w;
    o.k = 0;
    o.c_in = o.c_ring = o.c_out = o.u_in = o.u_disc = 0.f;
    const float tot = tot_h + tot_l;
    if (!(tot > 0.f)) return o;                  // fallback radius: no dependence
    // candidate from the start-up radius: r50 = (k-1) + frac, frac in (0, 1]
    int k = r50_hint > 0.5f ? static_cast<int>(ceilf(r50_hint)) : 0;
    for (int tries = 0; tries < 8; ++tries) {
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        const float km2 = static_cast<float>((k - 1) * (k - 1)), k2 = static_cast<float>(k * k);
        const float pcf = static_cast<float>(o.pc), prf = static_cast<float>(o.pr);
        FWalk pw(lane, ix.w);
        int p0 = lane;
        for (; p0 < npix; p0 += 256) {
            // eight loads in flight per lane; the stamp is still in L1 or L2
            float v[8], uu[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int p = p0 + 32 * u;
                v[u] = p < npix ? load_pix<DT>(a, ix.offset + p, sc) : 0.f;
                if (JVP) uu[u] = p < npix ? __ldg(a.tangent + ix.offset + p) : 0.f;
            }
            float ph[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float dj = pw.c - pcf, di = pw.r - prf;
                const float d2 = fmaf(di, di, dj * dj);      // an exact integer
                pw.next();
                const bool in0 = k >= 1 && d2 <= km2, in1 = d2 <= k2;   // zero-filled past the end
                ph[0] += in0 ? v[u] : 0.f;
                ph[1] += in1 ? v[u] : 0.f;
                if (JVP) {
                    ph[2] += in0 ? uu[u] : 0.f;
                    ph[3] += in1 ? uu[u] : 0.f;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) df_add(h[i], l[i], ph[i]);
        }
        warp_allsum_df(h, l);
        // 2 E - tot in double-float: the sign decides the crossing
        const float d1 = (2.f * h[1] - tot_h) + (2.f * l[1] - tot_l);
        const float d0 = (2.f * h[0] - tot_h) + (2.f * l[0] - tot_l);
        if (d1 < 0.f) {
            ++k;
        } else if (k >= 1 && d0 >= 0.f) {
            --k;
        } else {
            o.k = k;
            o.on = 1;
            o.u_in = h[2] + l[2];
            o.u_disc = h[3] + l[3];
            if (k == 0) {
                // r50 = H / (2 S) with S the brightest pixel
                const float Sf = h[1] + l[1], H = 0.5f * tot;
                o.c_ring = 0.5f * (0.5f * Sf - H) / (Sf * Sf) * kInvSqrt2Ln2F;
                o.c_out = 0.25f / Sf * kInvSqrt2Ln2F;
            } else {
                // r50 = (k-1) + (H - P) / (S - P); the differences from the pair sums
                const float D = (h[1] - h[0]) + (l[1] - l[0]);
                const float HP = 0.5f * ((tot_h - 2.f * h[0]) + (tot_l - 2.f * l[0]));
                o.c_out = 0.5f / D * kInvSqrt2Ln2F;
                o.c_ring = (0.5f * D - HP) / (D * D) * kInvSqrt2Ln2F;
                o.c_in = -0.5f / D * kInvSqrt2Ln2F;
            }
            return o;
        }
    }
    return o;
}

// The moment terms of one pixel at t = (t1, t2): f = I W times the 15
// monomials of degree <= 4 into P; for the JVP, the tangent u W times the
// six of degree <= 2, and u itself, into PU.
template <bool JVP>
__device__ __forceinline__ void moment_terms(const Geom& q, float t1, float t2, float v, float uu, float (&P)[15],
                                             float (&PU)[7]) {
    const float R2 = fmaf(q.A, t1 * t1, fmaf(q.B, t2 * t2, -q.G4 * (t1 * t2)));
    const float W = ex2(R2 * q.cw);
    const float f = v * W;
    const float f1 = f * t1, f2 = f * t2;
    const float f11 = f1 * t1, f12 = f1 * t2, f22 = f2 * t2;
    const float f111 = f11 * t1, f112 = f11 * t2, f122 = f12 * t2, f222 = f22 * t2;
    P[mono(0, 0)] += f;
    P[mono(1, 0)] += f1;
    P[mono(0, 1)] += f2;
    P[mono(2, 0)] += f11;
    P[mono(1, 1)] += f12;
    P[mono(0, 2)] += f22;
    P[mono(3, 0)] += f111;
    P[mono(2, 1)] += f112;
    P[mono(1, 2)] += f122;
    P[mono(0, 3)] += f222;
    P[mono(4, 0)] = fmaf(f111, t1, P[mono(4, 0)]);
    P[mono(3, 1)] = fmaf(f111, t2, P[mono(3, 1)]);
    P[mono(2, 2)] = fmaf(f112, t2, P[mono(2, 2)]);
    P[mono(1, 3)] = fmaf(f122, t2, P[mono(1, 3)]);
    P[mono(0, 4)] = fmaf(f222, t2, P[mono(0, 4)]);
    if (JVP) {
        const float h = uu * W;
        const float h1 = h * t1, h2 = h * t2;
        PU[0] += h;
        PU[1] += h1;
        PU[2] += h2;
        PU[3] = fmaf(h1, t1, PU[3]);
        PU[4] = fmaf(h1, t2, PU[4]);
        PU[5] = fmaf(h2, t2, PU[5]);
        PU[6] += uu;
    }
}

// One warp per stamp.  JVP = true: dtheta along a.tangent; false: the pixel
// gradient for a.v.
template <int DT, bool JVP>
__global__ void __launch_bounds__(256, 2) moment_grad_kernel(MomentGradArgs a) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned sidx = 0;
        if (lane == 0) sidx = atomicAdd(a.queue, 1u);
        sidx = __shfl_sync(kFull, sidx, 0);
        if (sidx >= static_cast<unsigned long long>(a.count)) break;
        const int64_t si = static_cast<int64_t>(sidx);
        const fse_stamp ix = a.idx[si];
        const fse_result mom = a.moments[si];
        uint32_t status = 0;
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        if (ix.h < 1 || ix.w < 1 || npl > FSE_MAX_PIX) {
            if (lane == 0 && a.status) a.status[si] = FSE_ST_BAD_SIZE;
            if (JVP && lane < 5) a.dtheta[si * 5 + lane] = 0.f;
            continue;
        }
        const int npix = static_cast<int>(npl);
        if (!(mom.status & FSE_ST_MOM_CONVERGED)) status |= FSE_ST_MOM_FAILED;
        const bool ellip = (a.mode & FSE_MOM_ELLIP) != 0;
        const bool sig_held = (a.mode & FSE_MOM_SIGW_FIXED) || (mom.status & FSE_ST_SIGW_CLAMPED);
        const bool sig_r50 = !sig_held && (a.mode & FSE_MOM_SIGW_R50);
        const float sc = (DT == FSE_BF16 && a.scale) ? a.scale[si] : 1.f;
        Geom q;
        q.x0 = mom.x0;
        q.y0 = mom.y0;
        q.g1 = ellip ? mom.e1 : 0.f;
        q.g2 = ellip ? mom.e2 : 0.f;
        q.s = mom.sigma_w;
        {
            const float gg = q.g1 * q.g1 + q.g2 * q.g2;
            q.A = 1.f + gg - 2.f * q.g1;
            q.B = 1.f + gg + 2.f * q.g1;
            q.G4 = 4.f * q.g2;
            q.cw = -kLog2e / (2.f * q.s * q.s);
        }
        if (!(q.s > 0.f) || !isfinite(q.cw)) status |= FSE_ST_MOM_FAILED;
        bool finite = true;
        // pass 1: the 15 weighted moments; the tangent's weighted sums (JVP);
        // and, for the growth curve, the brightest pixel and the total
        float Mh[15], Ml[15], Uh[7], Ul[7];
#pragma unroll
        for (int i = 0; i < 15; ++i) Mh[i] = Ml[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) Uh[i] = Ul[i] = 0.f;
        // JVP: the brightest pixel and the total ride along the moments pass
        // (its one launch reads the stamp once); the VJP has them from the
        // ring launch
        const bool inl = JVP && sig_r50;
        float vmax = -INFINITY, th_ = 0.f, tl_ = 0.f;
        int imax = 0x7fffffff;
        if (status == 0) {
            FWalk pw(lane, ix.w);
            int p0 = lane;
            // eight pixels per lane per step, loads ahead of use; then the tail
            for (; p0 + 224 < npix; p0 += 256) {
                float P[15], PU[7], ptot = 0.f;
#pragma unroll
                for (int i = 0; i < 15; ++i) P[i] = 0.f;
#pragma unroll
                for (int i = 0; i < 7; ++i) PU[i] = 0.f;
                float v[8], uu[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    v[u] = load_pix<DT>(a, ix.offset + p0 + 32 * u, sc);
                    if (JVP) uu[u] = __ldg(a.tangent + ix.offset + p0 + 32 * u);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (JVP && inl) {
                        if (v[u] > vmax) { vmax = v[u]; imax = p0 + 32 * u; }
                        ptot += v[u];
                    }
                    moment_terms<JVP>(q, pw.c - q.x0, pw.r - q.y0, v[u], JVP ? uu[u] : 0.f, P, PU);
                    pw.next();
                }
#pragma unroll
                for (int i = 0; i < 15; ++i) df_add(Mh[i], Ml[i], P[i]);
                if (JVP) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) df_add(Uh[i], Ul[i], PU[i]);
                    if (inl) df_add(th_, tl_, ptot);
                }
            }
            {
                float P[15], PU[7], ptot = 0.f;
#pragma unroll
                for (int i = 0; i < 15; ++i) P[i] = 0.f;
#pragma unroll
                for (int i = 0; i < 7; ++i) PU[i] = 0.f;
                for (int p = p0; p < npix; p += 32) {
                    const float v = load_pix<DT>(a, ix.offset + p, sc);
                    const float uu = JVP ? __ldg(a.tangent + ix.offset + p) : 0.f;
                    if (JVP && inl) {
                        if (v > vmax) { vmax = v; imax = p; }
                        ptot += v;
                    }
                    moment_terms<JVP>(q, pw.c - q.x0, pw.r - q.y0, v, uu, P, PU);
                    pw.next();
                }
#pragma unroll
                for (int i = 0; i < 15; ++i) df_add(Mh[i], Ml[i], P[i]);
                if (JVP) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) df_add(Uh[i], Ul[i], PU[i]);
                    if (inl) df_add(th_, tl_, ptot);
                }
            }
            // a NaN or Inf pixel (or tangent) makes I W (u W) non-finite
            // whatever its weight, and with it the warp's total
            float chk = (Mh[0] + Ml[0]) + (JVP ? Uh[6] + Uh[0] : 0.f) + (inl ? th_ : 0.f);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) chk += __shfl_xor_sync(kFull, chk, off);
            finite = isfinite(chk);
        }
        if (!finite) status |= FSE_ST_NONFINITE;
        float Su[7];
        if (status == 0) {
            warp_allsum_df(Mh, Ml);
            if (JVP) {
                warp_allsum_df(Uh, Ul);
#pragma unroll
                for (int i = 0; i < 7; ++i) Su[i] = Uh[i] + Ul[i];
            }
        }
        // the growth curve's crossing ring and constants, from the ring launch
        R50Grad rg;
        rg.on = 0;
        rg.pr = rg.pc = rg.k = 0;
        rg.c_in = rg.c_ring = rg.c_out = rg.u_in = rg.u_disc = 0.f;
        if (status == 0 && sig_r50) {
            if constexpr (JVP) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float ov = __shfl_xor_sync(kFull, vmax, off);
                    const int oi = __shfl_xor_sync(kFull, imax, off);
                    if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
                }
                float t2h[1] = {th_}, t2l[1] = {tl_};
                warp_allsum_df(t2h, t2l);
                rg = r50_ring<DT, JVP>(a, ix, npix, sc, mom.r50, imax, t2h[0], t2l[0], lane);
            } else {
                rg = a.r50g[si];
            }
        }
        // J: lane 5k + l assembles J_kl; then every lane holds all 25
        float X[25], xs[5], rhs[5];
        bool solved = false;
        float Jcol4[5];
        if (status == 0) {
            const int k = lane < 25 ? lane / 5 : 0, l = lane < 25 ? lane - 5 * (lane / 5) : 0;
            const float mine = jac_entry(q, k, l, Mh, Ml);
#pragma unroll
            for (int i = 0; i < 25; ++i) X[i] = __shfl_sync(kFull, mine, i);
#pragma unroll
            for (int i = 0; i < 5; ++i) Jcol4[i] = X[i * 5 + 4];
            // held parameters: rows and columns of a diagonal entry as large
            // as the active block's largest, with a zero right-hand side
            bool act[5] = {true, true, ellip, ellip, !(sig_held || sig_r50)};
            float big = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i)
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (act[i] && act[j]) big = fmaxf(big, fabsf(X[i * 5 + j]));
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                if (!act[i]) {
#pragma unroll
                    for (int j = 0; j < 5; ++j) X[i * 5 + j] = X[j * 5 + i] = 0.f;
                    X[i * 5 + i] = big;
                }
            }
            if (JVP) {
                // rhs = -(sum u psi + J_as dsigma_w); psi_k = W m_k
                float dsw = 0.f;
                if (rg.on)
                    dsw = rg.c_out * Su[6] + (rg.c_ring - rg.c_out) * rg.u_disc + (rg.c_in - rg.c_ring) * rg.u_in;
                const float ew1 = 2.f * q.g1 / (1.f + q.g1 * q.g1 + q.g2 * q.g2);
                const float ew2 = 2.f * q.g2 / (1.f + q.g1 * q.g1 + q.g2 * q.g2);
                float S5[5];
                S5[0] = Su[1];
                S5[1] = Su[2];
                S5[2] = (1.f - ew1) * Su[3] - (1.f + ew1) * Su[5];
                S5[3] = 2.f * Su[4] - ew2 * (Su[3] + Su[5]);
                S5[4] = q.A * Su[3] - q.G4 * Su[4] + q.B * Su[5] - q.s * q.s * Su[0];
#pragma unroll
                for (int i = 0; i < 5; ++i) rhs[i] = act[i] ? -(S5[i] + Jcol4[i] * dsw) : 0.f;
                solved = solve5(X, rhs, xs);
                if (solved && rg.on) xs[4] = dsw;
            } else {
                // transpose for J^T lambda = v
#pragma unroll
                for (int i = 0; i < 5; ++i)
#pragma unroll
                    for (int j = i + 1; j < 5; ++j) {
                        const float t = X[i * 5 + j];
                        X[i * 5 + j] = X[j * 5 + i];
                        X[j * 5 + i] = t;
                    }
#pragma unroll
                for (int i = 0; i < 5; ++i) rhs[i] = act[i] ? a.v[si * 5 + i] : 0.f;
                solved = solve5(X, rhs, xs);
            }
            if (!solved) status |= FSE_ST_FIT_SINGULAR;
        }
        if (JVP) {
            float val = 0.f;
#pragma unroll
            for (int i = 0; i < 5; ++i)
                if (lane == i && status == 0) val = xs[i];
            if (lane < 5) a.dtheta[si * 5 + lane] = val;
        } else {
            // dL/dI_p = -W(p) sum_k lambda_k m_k(p) + kappa d sigma_w / d I_p:
            // the per-stamp coefficients, for the write kernel
            VjpCoef cf;
            cf.x0 = q.x0;
            cf.y0 = q.y0;
            cf.A = q.A;
            cf.B = q.B;
            cf.G4 = q.G4;
            cf.cw = q.cw;
#pragma unroll
            for (int i = 0; i < 6; ++i) cf.c[i] = 0.f;
            cf.kc_in = cf.kc_ring = cf.kc_out = 0.f;
            cf.pc = static_cast<float>(rg.pc);
            cf.pr = static_cast<float>(rg.pr);
            cf.km2 = rg.k >= 1 ? static_cast<float>((rg.k - 1) * (rg.k - 1)) : -1.f;
            cf.k2 = static_cast<float>(rg.k * rg.k);
            cf.ring = rg.on && status == 0;
            cf.ok = status == 0;
            if (status == 0) {
                const float gg = q.g1 * q.g1 + q.g2 * q.g2;
                const float ew1 = 2.f * q.g1 / (1.f + gg), ew2 = 2.f * q.g2 / (1.f + gg);
                cf.c[0] = -xs[4] * q.s * q.s;
                cf.c[1] = xs[0];
                cf.c[2] = xs[1];
                cf.c[3] = xs[2] * (1.f - ew1) - xs[3] * ew2 + xs[4] * q.A;
                cf.c[4] = 2.f * xs[3] - xs[4] * q.G4;
                cf.c[5] = -xs[2] * (1.f + ew1) - xs[3] * ew2 + xs[4] * q.B;
                if (rg.on) {
                    float kappa = a.v[si * 5 + 4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) kappa = fmaf(-xs[i], Jcol4[i], kappa);
                    cf.kc_in = kappa * rg.c_in;
                    cf.kc_ring = kappa * rg.c_ring;
                    cf.kc_out = kappa * rg.c_out;
                }
            }
            if (lane == 0) a.coef[si] = cf;
        }
        if (lane == 0 && a.status) a.status[si] = status;
    }
}

// The growth curve of the start-up for the VJP's sigma_w derivative, in a
// launch of its own (the analysis kernel's body is long enough that its warps
// wait on instruction fetch; the JVP keeps it in its one kernel, whose passes
// then read the stamp from DRAM once): per stamp, one pass for the brightest
// pixel (ties to the lowest index) and the double-float total, then
// r50_ring's disc sums; the record goes to a.r50g for the analysis kernel.  One warp per stamp, stamps
// in grid-stride order; a stamp whose sigma_w does not come from the growth
// curve, or that the analysis kernel skips, gets on = 0.
template <int DT, bool JVP>
__global__ void __launch_bounds__(256) moment_r50_kernel(MomentGradArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t si = gw; si < a.count; si += nw) {
        const fse_stamp ix = a.idx[si];
        const fse_result mom = a.moments[si];
        R50Grad rg;
        rg.on = 0;
        rg.pr = rg.pc = rg.k = 0;
        rg.c_in = rg.c_ring = rg.c_out = rg.u_in = rg.u_disc = 0.f;
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        const bool sig_held = (a.mode & FSE_MOM_SIGW_FIXED) || (mom.status & FSE_ST_SIGW_CLAMPED);
        const bool use = ix.h >= 1 && ix.w >= 1 && npl <= FSE_MAX_PIX && (mom.status & FSE_ST_MOM_CONVERGED) &&
                         !sig_held && (a.mode & FSE_MOM_SIGW_R50);
        if (use) {
            const int npix = static_cast<int>(npl);
            const float sc = (DT == FSE_BF16 && a.scale) ? a.scale[si] : 1.f;
            float vmax = -INFINITY;
            int imax = 0x7fffffff;
            float th[1] = {0.f}, tl[1] = {0.f};
            int p0 = lane;
            for (; p0 + 224 < npix; p0 += 256) {
                float v[8], pt = 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = load_pix<DT>(a, ix.offset + p0 + 32 * u, sc);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (v[u] > vmax) { vmax = v[u]; imax = p0 + 32 * u; }
                    pt += v[u];
                }
                df_add(th[0], tl[0], pt);
            }
            {
                float pt = 0.f;
                for (int p = p0; p < npix; p += 32) {
                    const float v = load_pix<DT>(a, ix.offset + p, sc);
                    if (v > vmax) { vmax = v; imax = p; }
                    pt += v;
                }
                df_add(th[0], tl[0], pt);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float ov = __shfl_xor_sync(kFull, vmax, off);
                const int oi = __shfl_xor_sync(kFull, imax, off);
                if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
            }
            warp_allsum_df(th, tl);
            // a non-finite pixel leaves the total non-finite: no dependence
            // (the analysis kernel flags the stamp)
            if (isfinite(th[0]) && imax < npix)
                rg = r50_ring<DT, JVP>(a, ix, npix, sc, mom.r50, imax, th[0], tl[0], lane);
        }
        if (lane == 0) a.r50g[si] = rg;
    }
}

// The VJP's pixel gradient from the per-stamp coefficients: it depends on
// the pixels only through the coefficients, so this pass reads none and
// streams the writes.  One warp per stamp, stamps in grid-stride order;
// stamps of invalid size are left unwritten, like the analysis kernel
// leaves them; a stamp without a solution gets zeros.
__global__ void __launch_bounds__(256) moment_vjp_write_kernel(MomentGradArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t si = gw; si < a.count; si += nw) {
        const fse_stamp ix = a.idx[si];
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        if (ix.h < 1 || ix.w < 1 || npl > FSE_MAX_PIX) continue;
        const int npix = static_cast<int>(npl);
        const VjpCoef cf = a.coef[si];
        float* out = a.dpix + ix.offset;
        if (!cf.ok) {
            for (int p = lane; p < npix; p += 32) __stcs(out + p, 0.f);
            continue;
        }
        FWalk pw(lane, ix.w);
        for (int p = lane; p < npix; p += 32) {
            const float t1 = pw.c - cf.x0, t2 = pw.r - cf.y0;
            const float R2 = fmaf(cf.A, t1 * t1, fmaf(cf.B, t2 * t2, -cf.G4 * (t1 * t2)));
            const float W = ex2(R2 * cf.cw);
            const float Q = fmaf(t1, fmaf(cf.c[3], t1, fmaf(cf.c[4], t2, cf.c[1])),
                                 fmaf(t2, fmaf(cf.c[5], t2, cf.c[2]), cf.c[0]));
            float g = -W * Q;
            if (cf.ring) {
                const float dj = pw.c - cf.pc, di = pw.r - cf.pr;
                const float d2 = fmaf(di, di, dj * dj);
                g += d2 <= cf.km2 ? cf.kc_in : (d2 <= cf.k2 ? cf.kc_ring : cf.kc_out);
            }
            pw.next();
            __stcs(out + p, g);
        }
    }
}

template <int DT, bool JVP>
cudaError_t launch_t(const MomentGradArgs& a, cudaStream_t stream) {
    auto kern = moment_grad_kernel<DT, JVP>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if constexpr (!JVP) {
        if (a.mode & FSE_MOM_SIGW_R50) {
            long long rgrid = (a.count + 7) / 8;          // eight stamps (warps) per CTA
            const long long rcap = static_cast<long long>(sms) * 8;
            if (rgrid > rcap) rgrid = rcap;
            moment_r50_kernel<DT, false><<<static_cast<unsigned>(rgrid), 256, 0, stream>>>(a);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = static_cast<long long>(per_sm) * sms;
    const long long need = (a.count + 7) / 8;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 256, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess || JVP) return e;
    long long wgrid = (a.count + 7) / 8;          // eight stamps (warps) per CTA
    const long long wcap = static_cast<long long>(sms) * 8;
    if (wgrid > wcap) wgrid = wcap;
    moment_vjp_write_kernel<<<static_cast<unsigned>(wgrid), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_moment_grad(const MomentGradArgs& a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    const bool jvp = a.tangent != nullptr;
    if (a.dtype == FSE_BF16) return jvp ? launch_t<FSE_BF16, true>(a, stream) : launch_t<FSE_BF16, false>(a, stream);
    return jvp ? launch_t<FSE_F32, true>(a, stream) : launch_t<FSE_F32, false>(a, stream);
}

}  // namespace fse
