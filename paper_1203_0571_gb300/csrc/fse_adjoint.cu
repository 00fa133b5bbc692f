// fse_adjoint.cu -- chi^2 of the elliptical Sérsic model (Eqs. 10, 11) at
// given parameters and its adjoint (the vector-Jacobian product with the
// parameters and the pixels), for fse_sersic_chi2_grad.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fse_device.cuh"
#include "fse_internal.h"

namespace fse {
namespace {

// ------------------------------------------------------------------ adjoint
// chi^2 (Eq. 11) of the elliptical Sérsic model (Eq. 10) at caller-given
// parameters p = (x0, y0, e1, e2, I0, r_e, n), and the vector-Jacobian product
// of the upstream gradient gout[s] with d chi^2 / dp and d chi^2 / dI (pixels).
// With residual r = m - I and weights w:
//   d chi^2/dp = 2 sum w r dm/dp,   d chi^2/dI_i = -2 w_i r_i,
// m = I0 E, E = exp(-b u), u = (r_s / r_e)^(1/n).  The centre and the
// ellipticity act through the Sérsic radius r_s = R(g) / (1 - |g|) (Eq. A1).
// In the principal frame of the ellipse (t_par along the major axis at angle
// phi, 2 phi = arg g; t_perp across it) the radius is
//   r_s^2 = t_par^2 + k^2 t_perp^2,   k = (1 + |g|) / (1 - |g|),
// and with g = |g| (cos 2phi, sin 2phi)
//   d r_s^2/dg1 = cos2phi K1 t_perp^2 + sin2phi K2 t_par t_perp,
//   d r_s^2/dg2 = sin2phi K1 t_perp^2 - cos2phi K2 t_par t_perp,
//   K1 = 4 (1 + |g|) / (1 - |g|)^3,   K2 = 4 / (1 - |g|)^2,
//   d r_s^2/dx0 = -2 (cos phi t_par - sin phi k^2 t_perp),
//   d r_s^2/dy0 = -2 (sin phi t_par + cos phi k^2 t_perp).
// This form has no cancellation: written through R^2 and 1 - |g| separately,
// the two parts of dr_s/dg cancel exactly along the major axis.  At g = 0 the
// derivative of |g| is taken as 0 (the kink), which leaves
// d r_s^2/dg = (2 (t2^2 - t1^2), -4 t1 t2).  dm/d(r_s^2) = -m b u / (2 n r_s^2).
// One warp per stamp; each pixel is used once, so it is read straight from
// global memory (the lanes take consecutive pixels: coalesced).
template <int DT, bool IVAR, bool GRAD, bool DPIX>
__global__ void __launch_bounds__(256) chi2_grad_kernel(GradArgs a) {
    const int lane = threadIdx.x & 31;
    const float n_lo = static_cast<float>(kBnLo + 2 * kBnStep);
    const float n_hi = static_cast<float>(kBnLo + (kBnNodes - 3) * kBnStep);
    for (;;) {
        unsigned sidx = 0;
        if (lane == 0) sidx = atomicAdd(a.queue, 1u);
        sidx = __shfl_sync(kFull, sidx, 0);
        if (sidx >= static_cast<unsigned long long>(a.count)) break;
        const int64_t si = static_cast<int64_t>(sidx);
        const fse_stamp ix = a.idx[si];
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        const bool size_ok = ix.h >= 1 && ix.w >= 1 && npl <= FSE_MAX_PIX;
        float p[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) p[i] = a.params[si * 7 + i];
        const float x0 = p[0], y0 = p[1], g1 = p[2], g2 = p[3], I0 = p[4], re = p[5], n = p[6];
        const float gabs = sqrtf(g1 * g1 + g2 * g2);
        bool ok = size_ok && re > 0.f && n >= n_lo && n <= n_hi && gabs < 1.f && isfinite(I0) &&
                  isfinite(x0) && isfinite(y0) && isfinite(re);
        const int npix = size_ok ? static_cast<int>(npl) : 0;
        const float gof = a.gout ? static_cast<float>(a.gout[si]) : 1.f;
        if (!ok) {
            // parameters outside the model's domain: NaN results, NaN pixel gradient
            if (lane == 0) {
                if (a.chi2) a.chi2[si] = NAN;
                if (GRAD && a.dparams)
#pragma unroll
                    for (int i = 0; i < 7; ++i) a.dparams[si * 7 + i] = NAN;
            }
            if (DPIX)
                for (int q = lane; q < npix; q += 32) a.dpix[ix.offset + q] = NAN;
            continue;
        }
        float b, db;
        bn_lookup_f(a.bnf, n, &b, &db);
        const float inv_n = 1.f / n;
        // principal frame: cos 2phi, sin 2phi, then cos phi, sin phi
        const float c2 = gabs > 0.f ? g1 / gabs : 1.f, s2 = gabs > 0.f ? g2 / gabs : 0.f;
        const float cph = sqrtf(fmaxf(0.5f * (1.f + c2), 0.f));
        const float sph = copysignf(sqrtf(fmaxf(0.5f * (1.f - c2), 0.f)), s2);
        const float kap = (1.f + gabs) / (1.f - gabs), kap2 = kap * kap;
        const float zg = gabs > 0.f ? 0.f : 1.f;            // the g = 0 convention
        const float c0 = log2f(re);                          // log2(r_s / r_e) = 0.5 log2 r_s^2 - c0
        const float nbl = -b * kLog2e;
        const float kn = b * static_cast<float>(kLn2) * inv_n * inv_n;   // dm/dn = m u (kn a - b')
        const float sc = (DT == FSE_BF16 && a.scale) ? a.scale[si] : 1.f;
        const float* pf = static_cast<const float*>(a.pix) + ix.offset;
        const __nv_bfloat16* pb = static_cast<const __nv_bfloat16*>(a.pix) + ix.offset;
        const float* iv = IVAR ? a.inv_var + ix.offset : nullptr;
        float* dp = DPIX ? a.dpix + ix.offset : nullptr;
        float ch[1] = {0.f}, cl[1] = {0.f};
        // S: sum c E, sum c m u, sum c m u (kn a - b'), and with q = c m u / r_s^2:
        // sum q t_par, sum q k^2 t_perp, sum q (t_perp^2 - zg t_par^2),
        // sum q t_par t_perp   (c = 2 w r, a = log2(r_s / r_e)).  The n term is
        // combined per pixel before it is summed, so its parts do not cancel.
        float S[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) S[i] = 0.f;
        // Each lane loads KB pixels (and weights) ahead of using them: the
        // kernel reads every byte once, so what bounds it is how many loads are
        // in flight.  Per lane the pixels are still taken in the order
        // q = lane, lane + 32, ..., so the sums do not change.
        constexpr int KB = 8;
        FWalk pw(lane, ix.w);
        for (int q0 = lane; q0 < npix; q0 += 32 * KB) {
            float fv[KB], wv[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                const int q = q0 + 32 * j;
                const bool in = q < npix;
                if (DT == FSE_BF16)
                    fv[j] = in ? __bfloat162float(pb[q]) * sc : 0.f;
                else
                    fv[j] = in ? __ldcs(pf + q) : 0.f;
                wv[j] = IVAR ? (in ? __ldcs(iv + q) : 0.f) : 1.f;
            }
            float cp = 0.f;   // this lane's chi^2 over the KB pixels, then one double-float add
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                const int q = q0 + 32 * j;
                if (q >= npix) continue;
                const float f = fv[j];
                const float t1 = pw.c - x0;
                const float t2 = pw.r - y0;
                pw.next();
                const float tpa = fmaf(t1, cph, t2 * sph);
                const float tpe = fmaf(t2, cph, -t1 * sph);
                const float kte = kap2 * tpe;
                const float r2 = fmaf(kte, tpe, tpa * tpa);
                float u = 0.f, av = 0.f;
                if (r2 > 0.f) {
                    // MUFU log2: absolute error ~2^-22, the size of the rounding of
                    // log2 r_s^2 itself at these magnitudes
                    av = fmaf(0.5f, __log2f(r2), -c0);
                    u = ex2(av * inv_n);
                }
                const float E = ex2(u * nbl);
                const float wgt = wv[j];
                // one rounding for the residual, and an uncontracted square, in
                // every instance of the kernel, so that chi^2 does not depend on
                // which outputs were requested
                const float res = fmaf(I0, E, -f);
                const float wr = wgt * res;
                cp += __fmul_rn(wr, res);
                if (GRAD) {
                    const float c = 2.f * wr;
                    if (DPIX) __stcs(dp + q, __fmul_rn(-c, gof));
                    const float cmu = c * (I0 * E) * u;
                    S[0] = fmaf(c, E, S[0]);
                    S[1] += cmu;
                    S[2] = fmaf(cmu, fmaf(kn, av, -db), S[2]);
                    const float qv = r2 > 0.f ? __fdividef(cmu, r2) : 0.f;
                    S[3] = fmaf(qv, tpa, S[3]);
                    S[4] = fmaf(qv, kte, S[4]);
                    S[5] = fmaf(qv, fmaf(-zg * tpa, tpa, tpe * tpe), S[5]);
                    S[6] = fmaf(qv, tpa * tpe, S[6]);
                }
            }
            df_add(ch[0], cl[0], cp);
        }
        warp_allsum_df(ch, cl);
        if (GRAD) warp_allsum(S);
        if (lane == 0) {
            if (a.chi2) a.chi2[si] = static_cast<double>(ch[0]) + static_cast<double>(cl[0]);
            if (GRAD && a.dparams) {
                const float kr = -0.5f * b * inv_n;       // c dm/d(r_s^2) = kr q
                const float om = 1.f / (1.f - gabs);
                const float K2 = 4.f * om * om, K1 = (1.f + gabs) * om * K2;
                // d chi^2/dp, then times the upstream gradient as the last rounding
                float d[7];
                d[0] = -2.f * kr * fmaf(cph, S[3], -sph * S[4]);
                d[1] = -2.f * kr * fmaf(sph, S[3], cph * S[4]);
                if (gabs > 0.f) {
                    d[2] = kr * fmaf(c2 * K1, S[5], s2 * K2 * S[6]);
                    d[3] = kr * fmaf(s2 * K1, S[5], -c2 * K2 * S[6]);
                } else {
                    d[2] = 2.f * kr * S[5];
                    d[3] = -4.f * kr * S[6];
                }
                d[4] = S[0];
                d[5] = b * inv_n / re * S[1];
                d[6] = S[2];
                float* o = a.dparams + si * 7;
#pragma unroll
                for (int i = 0; i < 7; ++i) o[i] = __fmul_rn(d[i], gof);
            }
        }
    }
}

template <int DT, bool IVAR, bool GRAD, bool DPIX>
cudaError_t launch_grad_t(const GradArgs& a, cudaStream_t stream) {
    auto kern = chi2_grad_kernel<DT, IVAR, GRAD, DPIX>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = static_cast<long long>(per_sm) * sms;
    const long long need = (a.count + 7) / 8;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

template <int DT, bool IVAR>
cudaError_t launch_grad_dt(const GradArgs& a, cudaStream_t stream) {
    if (a.dpix) return launch_grad_t<DT, IVAR, true, true>(a, stream);
    if (a.dparams) return launch_grad_t<DT, IVAR, true, false>(a, stream);
    return launch_grad_t<DT, IVAR, false, false>(a, stream);
}

}  // namespace

cudaError_t launch_chi2_grad(const GradArgs& a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    if (!a.bnf) return cudaErrorInvalidValue;
    const bool iv = a.inv_var != nullptr;
    if (a.dtype == FSE_BF16)
        return iv ? launch_grad_dt<FSE_BF16, true>(a, stream) : launch_grad_dt<FSE_BF16, false>(a, stream);
    return iv ? launch_grad_dt<FSE_F32, true>(a, stream) : launch_grad_dt<FSE_F32, false>(a, stream);
}

}  // namespace fse
