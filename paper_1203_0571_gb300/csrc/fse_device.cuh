// fse_device.cuh -- device helpers shared by the estimator (fse_kernels.cu)
// and the chi^2 adjoint (fse_adjoint.cu): MUFU exp2, double-float
// accumulation, warp reductions, the strided pixel walk and the fp32 b(n)
// lookup.  Internal; each translation unit gets its own copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fse_internal.h"

namespace fse {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLog2e = 1.4426950408889634f;
constexpr double kLn2 = 0.6931471805599453;

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Double-float accumulation: (hi, lo) += b, carrying the exact rounding error
// of hi + b (Knuth's two-sum) in lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += e;
}

// ------------------------------------------------------------------ reductions
template <int N>
__device__ __forceinline__ void warp_allsum(float (&v)[N]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(kFull, v[i], off);
    }
}

__device__ __forceinline__ long long warp_allsum_ll(long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Sum of (hi, lo) pairs over the warp.  Both partners of a butterfly form
// hi + other.hi and its exact error in the same way, so every lane ends with
// the same pair.
template <int N>
__device__ __forceinline__ void warp_allsum_df(float (&hi)[N], float (&lo)[N]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float oh = __shfl_xor_sync(kFull, hi[i], off);
            const float ol = __shfl_xor_sync(kFull, lo[i], off);
            const float s = hi[i] + oh;
            const float bb = s - hi[i];
            const float e = (hi[i] - (s - bb)) + (oh - bb);
            lo[i] = (lo[i] + ol) + e;
            hi[i] = s;
        }
    }
}

// Pixel iterator: thread t handles p = t, t + nt, ... of a w-wide stamp.
struct PixelWalk {
    int row, col, dr, dc, w;
    __device__ PixelWalk(int t, int w_, int nt = 32) : w(w_) {
        row = t / w;
        col = t - row * w;
        dr = nt / w;
        dc = nt - dr * w;
    }
    __device__ __forceinline__ void next() {
        col += dc;
        row += dr;
        if (col >= w) {
            col -= w;
            ++row;
        }
    }
};

// Pixel coordinates of p = t, t + 32, ... of a w-wide stamp as floats.  They
// are integers, so every step is exact, and so is t = coordinate - centre.
struct FWalk {
    float c, r, dc, dr, wf;
    __device__ FWalk(int t, int w) {
        const int row = t / w;
        c = static_cast<float>(t - row * w);
        r = static_cast<float>(row);
        dr = static_cast<float>(32 / w);
        dc = static_cast<float>(32 - (32 / w) * w);
        wf = static_cast<float>(w);
    }
    __device__ __forceinline__ void next() {
        c += dc;
        r += dr;
        if (c >= wf) {
            c -= wf;
            r += 1.f;
        }
    }
};

// b(n), b'(n) in fp32 from a table of (b, b') at n = kBnLo + k kBnStep:
// cubic Hermite interpolation for b; b' as the linear interpolation of the
// node values of b' (error O(h^2 b''') ~ 1e-9).  Differentiating the
// interpolant of b instead would difference node values of b that carry fp32
// rounding, which the division by the step amplifies to ~1e-4.
__device__ __forceinline__ void bn_lookup_f(const float2* __restrict__ tab, float n, float* b,
                                            float* db) {
    const float x = (n - static_cast<float>(kBnLo)) * static_cast<float>(1.0 / kBnStep);
    int k = static_cast<int>(floorf(x));
    k = k < 0 ? 0 : (k > kBnNodes - 2 ? kBnNodes - 2 : k);
    const float t = x - static_cast<float>(k);
    const float2 p0 = tab[k], p1 = tab[k + 1];
    const float h = static_cast<float>(kBnStep);
    const float t2 = t * t, t3 = t2 * t;
    *b = p0.x + t2 * (3.f - 2.f * t) * (p1.x - p0.x) + (t3 - 2.f * t2 + t) * h * p0.y +
         (t3 - t2) * h * p1.y;
    *db = fmaf(t, p1.y - p0.y, p0.y);
}

}  // namespace
}  // namespace fse
