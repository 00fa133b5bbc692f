// fse_cutout.cu -- the cut-out of Sec. 4.1: from each large image, the
// square of side side_factor * r50 (six in the paper) around the brightest
// pixel, r50 from the growth curve around that pixel.  The cut-outs are
// packed back to back into a stamp buffer with its fse_stamp index, ready for
// the estimator.
//
// Three launches:
//   cutout_measure_kernel  one cluster of 8 CTAs per image, each over an
//                          eighth of its pixels: brightest pixel (ties to the
//                          lowest row-major index), the growth curve as exact
//                          64-bit fixed-point ring histograms in shared
//                          memory (the sums do not depend on their order),
//                          merged through distributed shared memory; r50 and
//                          the square, cut to the image;
//   cutout_scan_kernel     one CTA: exclusive prefix sum of h * w into the
//                          offsets of the packed buffer;
//   cutout_copy_kernel     one CTA per cut-out, a warp per row, lane loads.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cooperative_groups.h>

#include "fse_device.cuh"
#include "fse_internal.h"

namespace cg = cooperative_groups;

namespace fse {
namespace {

constexpr int kCutThreads = 256;
constexpr int kCutWarps = kCutThreads / 32;
constexpr int kCutCluster = 8;   // CTAs per image (a portable cluster size)
// Rings of the growth-curve histogram; a crossing beyond the last ring (r50
// above 2047 px) takes the largest side and reports r50 = NaN.
constexpr int kRings = 2048;
constexpr double kSqrt2Ln2D = 1.1774100225154747;

template <int DT>
__device__ __forceinline__ float img_pix(const CutoutArgs& a, int64_t off, float sc) {
    return DT == FSE_BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.images)[off]) * sc
                          : __ldg(static_cast<const float*>(a.images) + off);
}

// The ring k = ceil(sqrt(d2)) of a squared distance d2 < 2^31, with one MUFU
// operation: sqrt.approx of the float nearest d2 is within about 2^-22
// relative of the root, under 0.012 for roots up to 46341, so it truncates to
// c - 2, c - 1 or c, c the ceiling; two conditional increments give c (k * k
// stays below 2^32).
__device__ __forceinline__ unsigned ring_ceil32(unsigned d2) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(__uint2float_rn(d2)));
    unsigned k = __float2uint_rz(r);
    k += k * k < d2 ? 1u : 0u;
    k += k * k < d2 ? 1u : 0u;
    return k;
}

// Adds q to hist[key] for every lane with key >= 0.  Lanes of a warp stand on
// consecutive pixels, so neighbours usually share a ring: each run of equal
// keys in lane order is summed first (a segmented scan), and only its last
// lane adds to shared memory.  Far from the brightest pixel a row segment of
// 32 pixels spans a few rings, so this turns 32 colliding atomics into a few
// on distinct addresses.  The sums are integers, so the result does not
// depend on the grouping.  Every lane of the warp must call it.
__device__ __forceinline__ void ring_add(unsigned long long* hist, int key, unsigned long long q, int lane) {
    const int prev = __shfl_up_sync(kFull, key, 1);
    int start = (lane == 0 || prev != key) ? lane : 0;     // lane of the nearest run head at or before
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, start, off);
        if (lane >= off) start = max(start, o);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFull, q, off);
        if (lane - off >= start) q += o;
    }
    const int next = __shfl_down_sync(kFull, key, 1);
    if (key >= 0 && (lane == 31 || next != key)) atomicAdd(&hist[key], q);
}

// One cluster of kCutCluster CTAs per image; CTA r takes the r-th of
// kCutCluster equal ranges of the image's pixels (row-major).  The brightest
// pixel and the total are combined across the cluster through distributed
// shared memory, in rank order, so every CTA holds the same values; the
// ring histograms of the CTAs are summed by CTA 0, which finds the crossing.
template <int DT>
__global__ void __cluster_dims__(kCutCluster, 1, 1) __launch_bounds__(kCutThreads, 4)
    cutout_measure_kernel(CutoutArgs a) {
    __shared__ unsigned long long hist[kRings + 1];
    __shared__ float s_v[kCutWarps], s_amax[kCutWarps];
    __shared__ int s_i[kCutWarps];
    __shared__ int s_fin[kCutWarps];
    __shared__ long long s_tot[kCutWarps];
    // this CTA's part, read by the other CTAs of the cluster
    __shared__ float c_v, c_amax;
    __shared__ int c_i, c_fin;
    __shared__ long long c_tot;
    __shared__ int s_k;
    __shared__ long long s_prev, s_cur;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = static_cast<int>(cl.block_rank());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ncl = gridDim.x / kCutCluster;
    // every CTA of a cluster runs the same images and the same cluster
    // barriers: the loop bounds depend on the cluster alone
    for (int64_t img = blockIdx.x / kCutCluster; img < a.count; img += ncl) {
        const fse_stamp ix = a.img_idx[img];
        fse_cutout_info info = {0, 0, 0, 0, 0.f, 0u};
        const long long npl = static_cast<long long>(ix.h) * ix.w;
        const bool size_ok = ix.h >= 1 && ix.w >= 1 && npl <= (1LL << 28);
        const int npix = size_ok ? static_cast<int>(npl) : 0;
        const int lo = static_cast<int>(static_cast<long long>(npix) * rank / kCutCluster);
        const int hi = static_cast<int>(static_cast<long long>(npix) * (rank + 1) / kCutCluster);
        const float sc = (DT == FSE_BF16 && a.scale) ? a.scale[img] : 1.f;
        // pass 1: brightest pixel, largest |I|, finiteness
        float vmax = -INFINITY, amax = 0.f;
        int imax = 0x7fffffff;
        bool fin = true;
        for (int p0 = lo + tid; p0 < hi; p0 += 4 * kCutThreads) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * kCutThreads;
                v[u] = p < hi ? img_pix<DT>(a, ix.offset + p, sc) : -INFINITY;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * kCutThreads;
                if (p < hi) {
                    fin = fin && isfinite(v[u]);
                    if (v[u] > vmax) { vmax = v[u]; imax = p; }
                    amax = fmaxf(amax, fabsf(v[u]));
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ov = __shfl_xor_sync(kFull, vmax, off);
            const int oi = __shfl_xor_sync(kFull, imax, off);
            if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
            amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, off));
        }
        const bool wfin = __all_sync(kFull, fin);
        if (lane == 0) {
            s_v[warp] = vmax;
            s_i[warp] = imax;
            s_amax[warp] = amax;
            s_fin[warp] = wfin;
        }
        __syncthreads();
        if (tid == 0) {
            float bv = s_v[0], ba = s_amax[0];
            int bi = s_i[0], bf = s_fin[0];
            for (int k = 1; k < kCutWarps; ++k) {
                if (s_v[k] > bv || (s_v[k] == bv && s_i[k] < bi)) { bv = s_v[k]; bi = s_i[k]; }
                ba = fmaxf(ba, s_amax[k]);
                bf = bf && s_fin[k];
            }
            c_v = bv;
            c_i = bi;
            c_amax = ba;
            c_fin = bf;
        }
        cl.sync();   // every CTA's part of pass 1 is visible to the cluster
        vmax = *cl.map_shared_rank(&c_v, 0);
        imax = *cl.map_shared_rank(&c_i, 0);
        amax = *cl.map_shared_rank(&c_amax, 0);
        fin = *cl.map_shared_rank(&c_fin, 0);
#pragma unroll 1
        for (int r = 1; r < kCutCluster; ++r) {
            const float ov = *cl.map_shared_rank(&c_v, r);
            const int oi = *cl.map_shared_rank(&c_i, r);
            if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
            amax = fmaxf(amax, *cl.map_shared_rank(&c_amax, r));
            fin = fin && *cl.map_shared_rank(&c_fin, r);
        }
        const int pr = npix ? imax / ix.w : 0, pc = npix ? imax - (imax / ix.w) * ix.w : 0;
        // pass 2: ring histogram in fixed point, scale 2^S with amax * npix * 2^S < 2^62
        int e;
        frexpf(amax * static_cast<float>(npix), &e);
        int S = 62 - e;
        S = S > 100 ? 100 : (S < -100 ? -100 : S);
        const float fs = ldexpf(1.f, S);
        for (int k = tid; k <= kRings; k += kCutThreads) hist[k] = 0ull;
        __syncthreads();
        long long tot = 0;
        if (size_ok && fin) {
            // Each warp walks its own stretch of the CTA's range, so the warps
            // of a CTA stand rows apart, on different rings; the lanes take
            // consecutive pixels (one 128-byte load per warp and step), eight
            // loads in flight per lane.  The trip count is warp-uniform:
            // ring_add wants all 32 lanes.
            const int wch = (hi - lo + kCutWarps - 1) / kCutWarps;
            const int wlo = lo + warp * wch;
            const int whi = min(hi, wlo + wch);
            PixelWalk pw(wlo + lane, ix.w, 32);
            const bool narrow = ix.h <= 32768 && ix.w <= 32768;
            for (int b0 = wlo; b0 < whi; b0 += 8 * 32) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = b0 + u * 32 + lane;
                    v[u] = p < whi ? img_pix<DT>(a, ix.offset + p, sc) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    int key = -1;
                    unsigned long long qv = 0ull;
                    if (b0 + u * 32 + lane < whi) {
                        const long long q = __float2ll_rn(v[u] * fs);
                        tot += q;
                        qv = static_cast<unsigned long long>(q);
                        if (narrow) {   // both sides <= 32768: d2 < 2^31
                            const int di = pw.row - pr, dj = pw.col - pc;
                            const unsigned k = ring_ceil32(static_cast<unsigned>(di * di + dj * dj));
                            key = static_cast<int>(k < kRings ? k : kRings);
                        } else {
                            const long long di = pw.row - pr, dj = pw.col - pc;
                            const long long d2 = di * di + dj * dj;
                            long long k = static_cast<long long>(sqrtf(static_cast<float>(d2)));
                            while (k * k < d2) ++k;                   // k = ceil(sqrt(d2)): k-1 < d <= k,
                            while (k > 0 && (k - 1) * (k - 1) >= d2) --k;   // exact in integers
                            key = static_cast<int>(k < kRings ? k : kRings);
                        }
                    }
                    ring_add(hist, key, qv, lane);
                    pw.next();
                }
            }
        }
        tot = warp_allsum_ll(tot);
        if (lane == 0) s_tot[warp] = tot;
        __syncthreads();
        if (tid == 0) {
            long long t = 0;
            for (int k = 0; k < kCutWarps; ++k) t += s_tot[k];
            c_tot = t;
        }
        cl.sync();   // every CTA's histogram and total are complete
        if (rank == 0) {
            tot = 0;
#pragma unroll 1
            for (int r = 0; r < kCutCluster; ++r) tot += *cl.map_shared_rank(&c_tot, r);
            // the cluster's histogram, summed into this CTA's own (each ring by one thread)
            for (int k = tid; k <= kRings; k += kCutThreads) {
                unsigned long long t[kCutCluster];
#pragma unroll
                for (int r = 1; r < kCutCluster; ++r) t[r] = cl.map_shared_rank(hist, r)[k];   // all in flight
                unsigned long long s = hist[k];
#pragma unroll
                for (int r = 1; r < kCutCluster; ++r) s += t[r];
                hist[k] = s;
            }
            __syncthreads();
            // crossing ring: warp 0 scans the rings in lane chunks
            if (warp == 0) {
                constexpr int ch = (kRings + 1 + 31) / 32;
                const int k0 = lane * ch;
                long long own = 0;
                for (int k = k0; k < k0 + ch && k <= kRings; ++k) own += static_cast<long long>(hist[k]);
                long long incl = own;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const long long o2 = __shfl_up_sync(kFull, incl, off);
                    if (lane >= off) incl += o2;
                }
                long long run = incl - own;
                int kc = -1;
                long long prev = 0, cur = 0;
                for (int k = k0; k < k0 + ch && k < kRings; ++k) {   // the overflow ring is not a crossing
                    const long long nxt = run + static_cast<long long>(hist[k]);
                    if (2 * nxt >= tot) {
                        kc = k;
                        prev = run;
                        cur = nxt;
                        break;
                    }
                    run = nxt;
                }
                const unsigned hit = __ballot_sync(kFull, kc >= 0);
                const int src = hit ? __ffs(hit) - 1 : 0;
                kc = __shfl_sync(kFull, hit ? kc : -1, src);
                prev = __shfl_sync(kFull, prev, src);
                cur = __shfl_sync(kFull, cur, src);
                if (lane == 0) {
                    s_k = kc;
                    s_prev = prev;
                    s_cur = cur;
                }
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t st = 0;
                double r50;
                if (!size_ok) {
                    st = FSE_ST_BAD_SIZE;
                } else if (!fin) {
                    st = FSE_ST_NONFINITE;
                }
                if (st == 0) {
                    if (tot <= 0) {
                        st |= FSE_ST_INIT_FALLBACK;
                        r50 = kSqrt2Ln2D;
                    } else if (s_k < 0) {
                        r50 = NAN;                            // crossing beyond the last ring
                    } else if (s_k == 0) {
                        r50 = 0.25 * static_cast<double>(tot) / static_cast<double>(s_cur);
                    } else {
                        r50 = static_cast<double>(s_k - 1) +
                              static_cast<double>(tot - 2 * s_prev) / (2.0 * static_cast<double>(s_cur - s_prev));
                    }
                    long long side = isfinite(r50) ? static_cast<long long>(floor(a.side_factor * r50 + 0.5))
                                                   : static_cast<long long>(a.max_side);
                    side = side < a.min_side ? a.min_side : (side > a.max_side ? a.max_side : side);
                    int r0 = pr - static_cast<int>(side / 2), c0 = pc - static_cast<int>(side / 2);
                    int r1 = r0 + static_cast<int>(side), c1 = c0 + static_cast<int>(side);
                    r0 = r0 < 0 ? 0 : r0;
                    c0 = c0 < 0 ? 0 : c0;
                    r1 = r1 > ix.h ? ix.h : r1;
                    c1 = c1 > ix.w ? ix.w : c1;
                    info.row0 = r0;
                    info.col0 = c0;
                    info.h = r1 - r0;
                    info.w = c1 - c0;
                    info.r50 = static_cast<float>(r50);
                }
                info.status = st;
                a.info[img] = info;
                fse_stamp o;
                o.offset = 0;
                o.h = info.h;
                o.w = info.w;
                a.out_idx[img] = o;
            }
        }
        // CTA 0 has read the other histograms; shared state is reused by the next image
        cl.sync();
    }
}

// Exclusive prefix sum of h * w over the cut-outs, in one CTA of 1024
// threads, chunk by chunk with a running carry.
__global__ void __launch_bounds__(1024) cutout_scan_kernel(fse_stamp* out_idx, int64_t count, int64_t* total) {
    __shared__ long long warp_sum[32];
    __shared__ long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += 1024) {
        const int64_t i = base + tid;
        const long long n = i < count ? static_cast<long long>(out_idx[i].h) * out_idx[i].w : 0;
        long long incl = n;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            long long ws = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long o = __shfl_up_sync(kFull, ws, off);
                if (lane >= off) ws += o;
            }
            warp_sum[lane] = ws;                      // inclusive over warps
        }
        __syncthreads();
        const long long before = carry + (warp ? warp_sum[warp - 1] : 0) + incl - n;
        if (i < count) out_idx[i].offset = before;
        __syncthreads();
        if (tid == 1023) carry = before + n;
        __syncthreads();
    }
    if (tid == 0) *total = carry;
}

// One CTA per cut-out: its warps take rows in turn, lanes along the row.  A
// cut-out that does not fit in the output gets FSE_ST_NO_ROOM and is not
// copied.
template <typename T>
__global__ void __launch_bounds__(256) cutout_copy_kernel(CutoutArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const T* src = static_cast<const T*>(a.images);
    T* dst = static_cast<T*>(a.out_pix);
    for (int64_t i = blockIdx.x; i < a.count; i += gridDim.x) {
        const fse_cutout_info info = a.info[i];
        const fse_stamp o = a.out_idx[i];
        const long long n = static_cast<long long>(o.h) * o.w;
        if (n == 0) continue;
        if (o.offset + n > a.out_capacity) {
            if (threadIdx.x == 0) a.info[i].status = info.status | FSE_ST_NO_ROOM;
            continue;
        }
        const fse_stamp im = a.img_idx[i];
        for (int r = warp; r < o.h; r += nwarp) {
            const T* s = src + im.offset + static_cast<int64_t>(info.row0 + r) * im.w + info.col0;
            T* d = dst + o.offset + static_cast<int64_t>(r) * o.w;
            for (int c = lane; c < o.w; c += 32) d[c] = s[c];
        }
    }
}

}  // namespace

cudaError_t launch_cutout(const CutoutArgs& a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // clusters of kCutCluster CTAs, one image per cluster at a time; twice as
    // many clusters as fit at once keep every SM busy to the end
    long long clusters = static_cast<long long>(sms) * 2;
    if (clusters > a.count) clusters = a.count;
    const long long grid = clusters * kCutCluster;
    if (a.dtype == FSE_BF16)
        cutout_measure_kernel<FSE_BF16><<<static_cast<unsigned>(grid), kCutThreads, 0, stream>>>(a);
    else
        cutout_measure_kernel<FSE_F32><<<static_cast<unsigned>(grid), kCutThreads, 0, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cutout_scan_kernel<<<1, 1024, 0, stream>>>(a.out_idx, a.count, a.out_total);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long cgrid = a.count;
    const long long cap = static_cast<long long>(sms) * 8;
    if (cgrid > cap) cgrid = cap;
    if (a.out_pix) {
        if (a.dtype == FSE_BF16)
            cutout_copy_kernel<__nv_bfloat16><<<static_cast<unsigned>(cgrid), 256, 0, stream>>>(a);
        else
            cutout_copy_kernel<float><<<static_cast<unsigned>(cgrid), 256, 0, stream>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace fse
