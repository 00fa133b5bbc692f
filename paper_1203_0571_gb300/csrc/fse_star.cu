// fse_star.cu -- star profiles of Sec. 4.2 from weighted radial moments, at
// the centre and ellipticity of the moment stage (Secs. 2-3).
//
// r is the semi-major-axis radius of Eq. A1, r = R(g) / (1 - |g|); the radial
// moments r_k = sum I W r^k over the pixels carry the axis ratio q of the
// elliptical coordinates, which cancels from every ratio.
//   Gaussian: W = exp(-r^2 / 2 s_w^2); sigma = sqrt(r2 / r0); s_w <- sigma to
//     its fixed point; I0 = r0 / (pi sigma^2 q).
//   Moffat: W = (1 + r^2 / r_dw^2)^-3; beta = 1 / (r4 r0 / (2 r2^2) - 1),
//     r_d = sqrt(r2 / r0 (beta + 1)); r_dw <- r_d; I0 = r0 (beta+2) / (pi r_d^2 q).
// One warp per stamp: the stamp is read once from HBM (coalesced lane loads)
// into shared memory, where the iteration makes its passes over it; sums are
// double-float, within a lane and across the warp (xor shuffles), so that the
// step that stops the iteration is not swamped by rounding: near tol_sig = 1e-6
// the Moffat step is within a few fp32 ulps of the beta-amplified rounding.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fse_device.cuh"
#include "fse_internal.h"

namespace fse {
namespace {

constexpr float kPiF = 3.14159265358979f;
constexpr float kSqrt2Ln2F = 1.17741002f;
constexpr float kLn2F = 0.693147181f;
constexpr float kWeightCutF = 7.4446500f;   // sqrt(80 ln 2): W = exp(-r^2/2 s_w^2) = 2^-40 at r = this s_w

__host__ __device__ inline size_t star_warp_bytes(int max_pix) {
    return static_cast<size_t>(max_pix) * sizeof(float2);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Weighted moments of one pixel: f = I W(r), adds f, f r^2 and (Moffat) f r^4
// to the partial sums.  c is -log2(e)/(2 s_w^2) (Gaussian) or 1/r_dw^2 (Moffat).
template <int PROF>
__device__ __forceinline__ void star_pixel(float2 v, float c, float& a0, float& a1, float& a2) {
    float W;
    if (PROF == FSE_STAR_GAUSS) {
        W = ex2(v.y * c);
    } else {
        const float iv = rcp_approx(fmaf(v.y, c, 1.f));
        W = iv * iv * iv;
    }
    const float f = v.x * W;
    const float fr = f * v.y;
    a0 += f;
    a1 += fr;
    if (PROF == FSE_STAR_MOFFAT) a2 = fmaf(fr, v.y, a2);
}

// One warp per stamp.  The stamp is staged once into shared memory as
// (I, r^2) pairs, r^2 = R(g)^2 / (1 - |g|)^2 at the fixed centre and
// ellipticity, so that each pass of the iteration reads one 8-byte word per
// pixel and evaluates only the weight.  A lane sums eight pixels in fp32 and
// adds the partial to a double-float accumulator.
template <int DT, int PROF>
__global__ void __launch_bounds__(256) star_kernel(StarArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float2* sp = reinterpret_cast<float2*>(smem + static_cast<size_t>(warp) * star_warp_bytes(a.max_pix));
    for (;;) {
        unsigned sidx = 0;
        if (lane == 0) sidx = atomicAdd(a.queue, 1u);
        sidx = __shfl_sync(kFull, sidx, 0);
        if (sidx >= static_cast<unsigned long long>(a.count)) break;
        const int64_t si = static_cast<int64_t>(sidx);
        const fse_stamp ix = a.idx[si];
        const fse_result mom = a.moments[si];
        fse_star_result res = {};
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        if (ix.h < 1 || ix.w < 1 || npl > a.max_pix) {
            res.status = FSE_ST_BAD_SIZE;
        } else if (!(mom.status & FSE_ST_MOM_CONVERGED)) {
            res.status = FSE_ST_MOM_FAILED;   // no centre and ellipticity to measure at
        }
        const int npix = static_cast<int>(npl);
        const float g1 = mom.e1, g2 = mom.e2;
        const float gg = g1 * g1 + g2 * g2, gabs = sqrtf(gg);
        const float om = 1.f / (1.f - gabs);
        if (res.status == 0) {
            // stage (I, r^2), pixels decoded to fp32
            const float A = 1.f + gg - 2.f * g1, B = 1.f + gg + 2.f * g1, G4 = 4.f * g2;
            const float inv1g2 = om * om;
            const float sc = (DT == FSE_BF16 && a.scale) ? a.scale[si] : 1.f;
            bool fin = true;
            FWalk pw(lane, ix.w);
            for (int p0 = lane; p0 < npix; p0 += 256) {
                // eight loads in flight per lane before any is used
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = p0 + 32 * u;
                    v[u] = 0.f;
                    if (p < npix)
                        v[u] = DT == FSE_BF16
                            ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.pix)[ix.offset + p]) * sc
                            : __ldg(static_cast<const float*>(a.pix) + ix.offset + p);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = p0 + 32 * u;
                    if (p < npix) {
                        const float t1 = pw.c - mom.x0;
                        const float t2 = pw.r - mom.y0;
                        pw.next();
                        const float R2 = fmaf(A, t1 * t1, fmaf(B, t2 * t2, -G4 * (t1 * t2)));
                        sp[p] = make_float2(v[u], fmaxf(R2, 0.f) * inv1g2);
                        fin = fin && isfinite(v[u]);
                    }
                }
            }
            __syncwarp();
            if (!__all_sync(kFull, fin)) res.status = FSE_ST_NONFINITE;
        }
        if (res.status == 0) {
            const float q = (1.f - gabs) / (1.f + gabs);
            // start: sigma_w of the moments in r units (a Moffat r_d is about
            // twice the half-light radius, 1.1774 sigma_w, for beta near 4)
            float sw = (PROF == FSE_STAR_GAUSS ? 1.f : 2.35f) * mom.sigma_w * om;
            float size = sw, beta = 0.f, r0 = 0.f;
            int it;
            for (it = 1; it <= a.max_iter; ++it) {
                float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
                const float isw2 = 1.f / (sw * sw);
                const float c = PROF == FSE_STAR_GAUSS ? -0.5f * kLog2e * isw2 : isw2;
                // The Gaussian weight: only the rows whose pixels can have
                // W >= 2^-40 (r^2 <= 80 ln 2 s_w^2, i.e. R(g)^2 <= that times
                // (1-|g|)^2, an ellipse within |t2| <= rho sqrt(A) / (1-|g|^2)),
                // with a row of margin; the rows left out add less than
                // 2^-40 |I| r^k each.  The Moffat weight falls as r^-6 and
                // takes every pixel.
                int p = lane, pend = npix;
                if (PROF == FSE_STAR_GAUSS) {
                    const float rho = kWeightCutF * sw * (1.f - gabs);
                    const float hy = fminf(rho * sqrtf(1.f + gg - 2.f * g1) / (1.f - gg) + 1.f, 4096.f);
                    const int r0 = max(0, static_cast<int>(floorf(mom.y0 - hy)));
                    const int r1 = min(ix.h - 1, static_cast<int>(ceilf(mom.y0 + hy)));
                    if (r1 >= r0 && hy > 0.f) {
                        p = r0 * ix.w + lane;
                        pend = (r1 + 1) * ix.w;
                    }
                }
                for (; p + 224 < pend; p += 256) {
                    // eight pixels in two interleaved fp32 chains
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        star_pixel<PROF>(sp[p + 32 * u], c, a0, a1, a2);
                        star_pixel<PROF>(sp[p + 32 * u + 32], c, b0, b1, b2);
                    }
                    df_add(hi[0], lo[0], a0 + b0);
                    df_add(hi[1], lo[1], a1 + b1);
                    if (PROF == FSE_STAR_MOFFAT) df_add(hi[2], lo[2], a2 + b2);
                }
                {
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                    for (; p < pend; p += 32) star_pixel<PROF>(sp[p], c, a0, a1, a2);
                    df_add(hi[0], lo[0], a0);
                    df_add(hi[1], lo[1], a1);
                    if (PROF == FSE_STAR_MOFFAT) df_add(hi[2], lo[2], a2);
                }
                if (PROF == FSE_STAR_GAUSS) {
                    float h2[2] = {hi[0], hi[1]}, l2[2] = {lo[0], lo[1]};
                    warp_allsum_df(h2, l2);
                    hi[0] = h2[0]; hi[1] = h2[1]; lo[0] = l2[0]; lo[1] = l2[1];
                } else {
                    warp_allsum_df(hi, lo);
                }
                r0 = hi[0] + lo[0];
                const float r2 = hi[1] + lo[1], r4 = hi[2] + lo[2];
                if (!(r0 > 0.f) || !(r2 > 0.f)) {
                    res.status |= FSE_ST_MOM_FAILED;
                    break;
                }
                const float ir0 = 1.f / r0;
                if (PROF == FSE_STAR_GAUSS) {
                    size = sqrtf(r2 * ir0);
                } else {
                    const float ratio = r4 * r0 / (2.f * r2 * r2);
                    if (!(ratio > 1.f)) {
                        res.status |= FSE_ST_MOM_FAILED;
                        break;
                    }
                    beta = 1.f / (ratio - 1.f);
                    size = sqrtf(r2 * ir0 * (beta + 1.f));
                }
                if (!isfinite(size) || !(size > 0.f)) {
                    res.status |= FSE_ST_MOM_FAILED;
                    break;
                }
                const float step = fabsf(__fdividef(size, sw) - 1.f);
                sw = size;
                if (step <= a.tol) {
                    res.status |= FSE_ST_MOM_CONVERGED;
                    break;
                }
            }
            if (it > a.max_iter) {
                res.status |= FSE_ST_MOM_MAXITER;
                it = a.max_iter;
            }
            res.iters = it;
            res.size = size;
            res.beta = beta;
            if (res.status & FSE_ST_MOM_CONVERGED) {
                // closed forms at the fixed point, from the last pass's r0
                if (PROF == FSE_STAR_GAUSS) {
                    res.I0 = r0 / (kPiF * size * size * q);
                    res.flux = 2.f * kPiF * size * size * res.I0 * q;
                    res.r50 = size * kSqrt2Ln2F;
                } else {
                    res.I0 = r0 * (beta + 2.f) / (kPiF * size * size * q);
                    res.flux = beta > 1.f ? kPiF * size * size * res.I0 * q / (beta - 1.f) : INFINITY;
                    // r50 = r_d sqrt(2^x - 1), x = 1/(beta-1): expm1 keeps the
                    // digits for large beta; for x > 60 the -1 is below rounding
                    // and 2^(x/2) stays finite up to x = 256
                    const float x = beta > 1.f ? 1.f / (beta - 1.f) : INFINITY;
                    res.r50 = x <= 60.f ? size * sqrtf(expm1f(x * kLn2F)) : size * exp2f(0.5f * x);
                }
            }
        }
        if (lane == 0) a.out[si] = res;
        __syncwarp();
    }
}

template <int DT, int PROF>
cudaError_t launch_star_t(const StarArgs& a, cudaStream_t stream) {
    auto kern = star_kernel<DT, PROF>;
    const size_t spw = star_warp_bytes(a.max_pix);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // shared memory bounds the resident warps: take the CTA size (8, 4, 2 or
    // 1 warps) with the most resident warps per SM
    int wpc = 0, per_sm = 0, best = 0;
    for (int c = 8; c >= 1; c >>= 1) {
        const size_t smem = spw * c;
        if (smem > 227 * 1024) continue;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * c, smem);
        if (e != cudaSuccess) return e;
        if (b * c > best) {
            best = b * c;
            wpc = c;
            per_sm = b;
        }
    }
    if (best < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = spw * wpc;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    long long grid = static_cast<long long>(per_sm) * sms;
    const long long need = (a.count + wpc - 1) / wpc;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 32 * wpc, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_star(const StarArgs& a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    if (a.dtype == FSE_BF16)
        return a.profile == FSE_STAR_MOFFAT ? launch_star_t<FSE_BF16, FSE_STAR_MOFFAT>(a, stream)
                                            : launch_star_t<FSE_BF16, FSE_STAR_GAUSS>(a, stream);
    return a.profile == FSE_STAR_MOFFAT ? launch_star_t<FSE_F32, FSE_STAR_MOFFAT>(a, stream)
                                        : launch_star_t<FSE_F32, FSE_STAR_GAUSS>(a, stream);
}

}  // namespace fse
