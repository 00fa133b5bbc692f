// fse_kernels.cu -- sm_103a kernels of the fast shape estimator
// (Li, Xin & Cui 2012): weighted-moment centroid (Sec. 2), KSB ellipticity
// with an elliptical weight (Sec. 3, Appendices A and B) and the Sérsic
// profile fit with I0 at its closed form (Sec. 4.1, Eqs. 10-13).
//
// Execution model: two persistent launches per batch (the start-up and moment
// iteration, then the fit); in each, every warp owns one stamp at a time
// and takes the next from an atomic work counter.  The stamp is staged once
// HBM -> shared memory (1-D TMA bulk copy for its 16-byte-aligned body, plain
// loads for the ragged ends) and every later pass (start-up, moment
// iterations, fit iterations) reads shared memory only.  Per pixel the work is
// fp32 (MUFU ex2 for the weight and the profile); per-lane partial sums are
// reduced with xor shuffles, which give every lane the same total, so all
// lanes run the scalar update redundantly and stay in lock-step.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "fse_device.cuh"
#include "fse_internal.h"

namespace fse {
namespace {

constexpr double kSqrt2Ln2 = 1.1774100225154747;   // half-light radius / sigma of a Gaussian
constexpr double kPi = 3.141592653589793;
constexpr unsigned kWaitLimit = 1u << 22;          // bounded mbarrier polls

// (b(n), b'(n)) at n_k = kBnLo + k kBnStep, built once per device in FP64;
// g_bnf holds the same nodes rounded to fp32 for the fit's per-iteration use.
__device__ double2 g_bn[kBnNodes];
__device__ float2 g_bnf[kBnNodes];

// ------------------------------------------------------------------ PTX
// 2^x to about one ulp, for the final refinement pass: x = k + f with k an
// integer and |f| <= 1/2, 2^f from the Taylor series of exp(f ln 2) to degree 7
// (truncation below 6e-9 relative), then the exponent raised by k.
__device__ __forceinline__ float exp2_acc(float x) {
    if (!(x >= -126.f)) return 0.f;
    if (x > 127.f) return INFINITY;
    const float k = rintf(x);
    const float f = x - k;
    // Horner's scheme (about 1.2 ulp; shorter-chain schemes round the leading
    // terms earlier and lose accuracy)
    float p = 1.5252733804059841e-05f;
    p = fmaf(p, f, 1.540353039338161e-04f);
    p = fmaf(p, f, 1.3333558146428443e-03f);
    p = fmaf(p, f, 9.618129107628477e-03f);
    p = fmaf(p, f, 5.550410866482158e-02f);
    p = fmaf(p, f, 2.4022650695910072e-01f);
    p = fmaf(p, f, 6.931471805599453e-01f);
    p = fmaf(p, f, 1.f);
    return __int_as_float(__float_as_int(p) + (static_cast<int>(k) << 23));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_bulk_load(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// ------------------------------------------------------------------ stamp groups
// NW warps may share one stamp (large stamps, whose shared-memory tile leaves
// room for few of them per SM).  Thread t = 32 (warp in group) + lane strides
// the pixels by 32 NW; reductions finish through the group's shared scratch in
// a fixed order, so every thread of the group ends with the same bits, and the
// scalar steps run redundantly in all of them, as in a single warp.  With
// NW = 1 every operation below is the single-warp one (shuffles, __syncwarp).
template <int NW>
struct Grp {
    static constexpr int NT = 32 * NW;
    int t;        // thread index in the group
    int lane;
    int wi;       // warp index in the group
    float* red;   // NW x 32 words of reduction scratch (NW > 1), 8-byte aligned
    int bar;      // named barrier of the group (NW > 1)

    __device__ __forceinline__ void sync() const {
        if (NW == 1)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(NT) : "memory");
    }

    template <int N>
    __device__ __forceinline__ void allsum(float (&v)[N]) const {
        static_assert(N <= 32, "reduction width");
        warp_allsum(v);
        if (NW > 1) {
            sync();   // the previous reduction's readers are done with red
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < N; ++i) red[wi * 32 + i] = v[i];
            }
            sync();
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float acc = red[i];
#pragma unroll
                for (int k = 1; k < NW; ++k) acc += red[k * 32 + i];
                v[i] = acc;
            }
        }
    }

    template <int N>
    __device__ __forceinline__ void allsum_df(float (&hi)[N], float (&lo)[N]) const {
        static_assert(2 * N <= 32, "reduction width");
        warp_allsum_df(hi, lo);
        if (NW > 1) {
            sync();
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    red[wi * 32 + i] = hi[i];
                    red[wi * 32 + N + i] = lo[i];
                }
            }
            sync();
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float h = red[i], l = red[N + i];
#pragma unroll
                for (int k = 1; k < NW; ++k) {
                    const float oh = red[k * 32 + i], ol = red[k * 32 + N + i];
                    const float sum = h + oh;
                    const float bb = sum - h;
                    const float e = (h - (sum - bb)) + (oh - bb);
                    l = (l + ol) + e;
                    h = sum;
                }
                hi[i] = h;
                lo[i] = l;
            }
        }
    }

    __device__ __forceinline__ long long allsum_ll(long long v) const {
        v = warp_allsum_ll(v);
        if (NW > 1) {
            long long* r = reinterpret_cast<long long*>(red);
            sync();
            if (lane == 0) r[wi * 16] = v;
            sync();
            long long acc = r[0];
#pragma unroll
            for (int k = 1; k < NW; ++k) acc += r[k * 16];
            v = acc;
        }
        return v;
    }

    __device__ __forceinline__ bool all(bool b) const {
        b = __all_sync(kFull, b);
        if (NW > 1) {
            sync();
            if (lane == 0) red[wi * 32] = b ? 1.f : 0.f;
            sync();
            bool acc = true;
#pragma unroll
            for (int k = 0; k < NW; ++k) acc = acc && red[k * 32] != 0.f;
            b = acc;
        }
        return b;
    }
};

// ------------------------------------------------------------------ b(n)
// Digamma for z > 0: recurrence up to z >= 10, then the asymptotic series
// psi(z) ~ ln z - 1/(2z) - sum B_2k / (2k z^2k) (Abramowitz & Stegun 6.3.18).
__device__ double digamma(double z) {
    double acc = 0.0;
    while (z < 10.0) {
        acc -= 1.0 / z;
        z += 1.0;
    }
    const double r = 1.0 / (z * z);
    const double tail =
        r * (1.0 / 12 - r * (1.0 / 120 - r * (1.0 / 252 - r * (1.0 / 240 - r * (1.0 / 132)))));
    return acc + log(z) - 0.5 / z - tail;
}

// P(a, x) (regularised lower incomplete gamma) and dP/da from the series
// P = sum_k T_k, T_k = x^(a+k) e^-x / Gamma(a+k+1), with
// dT_k/da = T_k (ln x - psi(a+k+1)) and psi(a+k+1) = psi(a+k) + 1/(a+k).
__device__ void gamma_p_series(double a, double x, double* P, double* dPda) {
    const double lx = log(x);
    double T = exp(a * lx - x - lgamma(a + 1.0));
    double psi = digamma(a + 1.0);
    double sum = T, dsum = T * (lx - psi);
    for (int k = 1; k < 4000; ++k) {
        T *= x / (a + k);
        psi += 1.0 / (a + k);
        sum += T;
        dsum += T * (lx - psi);
        if (T < 1e-18 * sum) break;
    }
    *P = sum;
    *dPda = dsum;
}

// b(n): Newton on P(2n, b) = 1/2 from the large-n expansion, kept inside the
// bracket (0, 2n) (the median of Gamma(2n) lies below its mean).  b'(n) by
// implicit differentiation: b' = -dP/dn / dP/db = -2 dP/da / (b^(a-1) e^-b / Gamma(a)).
__global__ void build_bn_kernel() {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kBnNodes) return;
    const double n = kBnLo + k * kBnStep;
    const double a = 2.0 * n;
    double lo = 0.0, hi = a;
    double b = a - 1.0 / 3.0 + 4.0 / (405.0 * n);
    if (!(b > lo && b < hi)) b = 0.5 * a;
    double P = 0.0, dPda = 0.0;
    for (int it = 0; it < 100; ++it) {
        gamma_p_series(a, b, &P, &dPda);
        const double f = P - 0.5;
        if (f > 0.0) hi = b; else lo = b;
        const double dPdx = exp((a - 1.0) * log(b) - b - lgamma(a));
        double nb = b - f / dPdx;
        if (!(nb > lo && nb < hi)) nb = 0.5 * (lo + hi);
        const bool done = fabs(nb - b) <= 4e-16 * b;
        b = nb;
        if (done) break;
    }
    gamma_p_series(a, b, &P, &dPda);
    const double dPdx = exp((a - 1.0) * log(b) - b - lgamma(a));
    const double db = -2.0 * dPda / dPdx;
    g_bn[k] = make_double2(b, db);
    g_bnf[k] = make_float2(static_cast<float>(b), static_cast<float>(db));
}

// Cubic Hermite interpolation of the table (b from b and b' at the nodes;
// b' as the derivative of that cubic).
__device__ __forceinline__ void bn_eval(double n, double* b, double* db) {
    double x = (n - kBnLo) * (1.0 / kBnStep);
    int k = static_cast<int>(floor(x));
    k = k < 0 ? 0 : (k > kBnNodes - 2 ? kBnNodes - 2 : k);
    const double t = x - k;
    const double2 p0 = g_bn[k], p1 = g_bn[k + 1];
    const double h = kBnStep;
    const double t2 = t * t, t3 = t2 * t;
    *b = (2 * t3 - 3 * t2 + 1) * p0.x + (t3 - 2 * t2 + t) * h * p0.y + (-2 * t3 + 3 * t2) * p1.x +
         (t3 - t2) * h * p1.y;
    *db = ((6 * t2 - 6 * t) * p0.x + (3 * t2 - 4 * t + 1) * h * p0.y + (-6 * t2 + 6 * t) * p1.x +
           (3 * t2 - 2 * t) * h * p1.y) /
          h;
}

// The same interpolation in fp32 from the rounded nodes (fit iterations).
__device__ __forceinline__ void bn_eval_f(float n, float* b, float* db) {
    bn_lookup_f(g_bnf, n, b, db);
}

// b''(n) as the slope of b' across the table interval (first-order accurate;
// it only enters the curvature term of the final Newton steps).
__device__ __forceinline__ float bn_d2_f(float n) {
    const float x = (n - static_cast<float>(kBnLo)) * static_cast<float>(1.0 / kBnStep);
    int k = static_cast<int>(floorf(x));
    k = k < 0 ? 0 : (k > kBnNodes - 2 ? kBnNodes - 2 : k);
    return (g_bnf[k + 1].y - g_bnf[k].y) * static_cast<float>(1.0 / kBnStep);
}

__global__ void eval_bn_kernel(const double* n, double* b, double* db, int64_t count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    double bb, dd;
    bn_eval(n[i], &bb, &dd);
    b[i] = bb;
    if (db) db[i] = dd;
}

// ------------------------------------------------------------------ per-warp layout
// [pixels: max_pix + 4 floats][aux: max(max_pix, 512) floats][ivar: max_pix + 4 (opt)][mbarrier]
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t pix_bytes(int max_pix) { return align16((size_t)(max_pix + 4) * 4); }
__host__ __device__ inline size_t aux_bytes(int max_pix) {
    return align16((size_t)(max_pix > 512 ? max_pix : 512) * 4);
}
__host__ __device__ inline size_t warp_bytes(int max_pix, bool ivar) {
    return pix_bytes(max_pix) + aux_bytes(max_pix) + (ivar ? pix_bytes(max_pix) : 0) + 16;
}
// Shared memory of a stamp group: the tile above plus, for nw > 1 warps per
// stamp, the reduction scratch (nw x 32 words) and the work-counter word.
__host__ __device__ inline size_t group_bytes(int max_pix, bool ivar, int nw) {
    return warp_bytes(max_pix, ivar) + (nw > 1 ? static_cast<size_t>(nw) * 128 + 16 : 0);
}

// Rings the start-up's growth curve can need for stamps of at most max_pix
// pixels and sides of at most FSE_MAX_SIDE: ring k holds the pixels at
// distance k-1 < d <= k from the brightest pixel, so a stamp needs rings 0 to
// ceil(corner distance) + 1 (the histogram's kmax), and the corner distance
// is at most that of the most elongated h x w with h w <= max_pix.
inline int ring_slots(int max_pix) {
    int best = 0;
    for (int h = 1; h <= FSE_MAX_SIDE; ++h) {
        int w = max_pix / h;
        if (w < 1) break;
        if (w > FSE_MAX_SIDE) w = FSE_MAX_SIDE;
        const int d = (h - 1) * (h - 1) + (w - 1) * (w - 1);
        if (d > best) best = d;
    }
    int k = 0;
    while (k * k < best) ++k;
    return k + 2;
}

// The moment stages keep a smaller tile: the pixels, and an auxiliary area
// only for the raw bf16 staging and, in the start-up launch, the ring
// histogram (three 32-bit words per ring); no inverse variance (the moments do
// not use it).  For 48x48 fp32 that is 9.2 KB per warp in the moment launch
// and 10.8 KB in the start-up, instead of the fit's 18.5 KB.
__host__ __device__ inline size_t aux_bytes_moments(int max_pix, bool bf16, int slots) {
    const size_t raw = bf16 ? static_cast<size_t>(max_pix + 8) * 2 : 0;
    const size_t hist = static_cast<size_t>(slots) * 12;
    return align16(raw > hist ? raw : hist);
}
__host__ __device__ inline constexpr bool moment_stage(int stage) {
    return stage == kStageCentroid || stage == kStageEllipticity || stage == kStageMoments ||
           stage == kStageStartup;
}
__host__ __device__ inline size_t stage_aux_bytes(int stage, int max_pix, bool bf16, int slots) {
    return moment_stage(stage) ? aux_bytes_moments(max_pix, bf16, stage == kStageStartup ? slots : 0)
                               : aux_bytes(max_pix);
}
__host__ __device__ inline size_t stage_warp_bytes(int stage, int max_pix, bool bf16, bool ivar, int slots) {
    return pix_bytes(max_pix) + stage_aux_bytes(stage, max_pix, bf16, slots) +
           (ivar && !moment_stage(stage) ? pix_bytes(max_pix) : 0) + 16;
}
__host__ __device__ inline size_t stage_group_bytes(int stage, int max_pix, bool bf16, bool ivar, int nw,
                                                    int slots) {
    return stage_warp_bytes(stage, max_pix, bf16, ivar, slots) +
           (nw > 1 ? static_cast<size_t>(nw) * 128 + 16 : 0);
}

// Stage a stamp (npix elements at gsrc) into shared memory.  The 16-byte
// aligned body moves with one bulk TMA copy completing on `bar`; the head
// and tail are loaded by lanes.  Returns false if the bounded wait expired.
// Floats: the stamp starts at buf + pad with pad chosen so that the body's
// shared address is 16-byte aligned too.  BF16: the raw 2-byte values are
// staged in `raw` first and decoded (times scale) into the float buffer.
template <int DT, int NW>
__device__ bool stage_stamp(float* buf, float** stamp, float* raw, const void* gsrc, int npix,
                            float scale, uint64_t* bar, uint32_t* phase, const Grp<NW>& g) {
    constexpr int NT = Grp<NW>::NT;
    constexpr int esz = DT == FSE_BF16 ? 2 : 4;
    const uintptr_t ga = reinterpret_cast<uintptr_t>(gsrc);
    int head = static_cast<int>(((16 - (ga & 15)) & 15) / esz);
    if ((ga & (esz - 1)) != 0) head = npix;          // not element aligned: no TMA
    if (head > npix) head = npix;
    constexpr int vec = 16 / esz;
    const int body = ((npix - head) / vec) * vec;
    const int tail = head + body;
    char* dst_base;
    int pad;
    if (DT == FSE_BF16) {
        // raw bf16 staging: element i at raw_bytes + 2*(pad + i), (pad + head) % 8 == 0
        pad = (8 - (head & 7)) & 7;
        dst_base = reinterpret_cast<char*>(raw);
        *stamp = buf;
    } else {
        pad = (4 - (head & 3)) & 3;
        dst_base = reinterpret_cast<char*>(buf);
        *stamp = buf + pad;
    }
    // order the group's earlier generic-proxy accesses to the buffer before
    // the async-proxy (TMA) write into it
    fence_proxy_async();
    g.sync();
    bool ok = true;
    if (body > 0) {
        if (g.t == 0) {
            mbar_expect_tx(bar, static_cast<uint32_t>(body * esz));
            tma_bulk_load(dst_base + (size_t)(pad + head) * esz,
                          static_cast<const char*>(gsrc) + (size_t)head * esz,
                          static_cast<uint32_t>(body * esz), bar);
        }
    }
    if (DT == FSE_BF16) {
        const __nv_bfloat16* gb = static_cast<const __nv_bfloat16*>(gsrc);
        __nv_bfloat16* r = reinterpret_cast<__nv_bfloat16*>(dst_base) + pad;
        for (int i = g.t; i < head; i += NT) r[i] = gb[i];
        for (int i = tail + g.t; i < npix; i += NT) r[i] = gb[i];
    } else {
        const float* gf = static_cast<const float*>(gsrc);
        float* s = *stamp;
        for (int i = g.t; i < head; i += NT) s[i] = __ldg(gf + i);
        for (int i = tail + g.t; i < npix; i += NT) s[i] = __ldg(gf + i);
    }
    if (body > 0) {
        ok = false;
        for (unsigned it = 0; it < kWaitLimit; ++it) {
            if (mbar_try_wait(bar, *phase & 1u)) {
                ok = true;
                break;
            }
        }
        ++*phase;
    }
    g.sync();   // the head and tail loads of the other threads are visible
    // every thread of the group waited on the same barrier; they act on one
    // verdict
    ok = g.all(ok);
    if (DT == FSE_BF16 && ok) {
        const __nv_bfloat16* r = reinterpret_cast<const __nv_bfloat16*>(dst_base) + pad;
        float* s = *stamp;
        for (int i = g.t; i < npix; i += NT) s[i] = __bfloat162float(r[i]) * scale;
    }
    g.sync();
    return ok;
}

// Model values above this many noise sigmas carry an fp32 rounding (6e-8 of the
// value) that is no longer small against the residual; the final refinement
// of the fit evaluates chi^2 for those pixels in fp64.
constexpr float kBrightSigma = 512.f;

// ------------------------------------------------------------------ moments
struct MomState {
    int xi, yi;      // integer part of the centre
    float xf, yf;    // fractional part, |.| <= 0.5 after renormalisation
    float g1, g2;    // weight ellipticity g_w
    float sw;        // weight size sigma_w
    int xr, yr;      // reference pixel of the stored per-pixel offsets
};

// The moment sums run over the pixels whose weight W = 2^(-R^2 log2(e) /
// (2 s_w^2)) is at least 2^-40, i.e. R^2 <= 80 ln 2 s_w^2: a pixel outside
// adds less than 2^-40 |I| |theta|^k to a sum, so all of them together move
// the centre by less than 2^-40 sum|I| max|theta| / sum I W (below 1e-9 px on
// the benchmark's faintest stamps) and g and s_w by as little.  The ellipse
// A t1^2 + B t2^2 - 4 g2 t1 t2 <= Rc^2 (Eq. A1; the determinant of the form
// is (1 - |g|^2)^2) lies inside |t1| <= Rc sqrt(B) / (1 - |g|^2), |t2| <=
// Rc sqrt(A) / (1 - |g|^2); the box adds a pixel of margin and is cut to the
// stamp.  Compact objects (stars, small galaxies) cover a fraction of their
// stamp, which is the work saved.
constexpr float kWeightCut = 7.4446500f;   // sqrt(80 ln 2)

struct Box {
    int r0, c0;   // first row and column
    int bh, bw;   // rows and columns (at least one each)
    // stamp index of the box's last pixel
    __device__ __forceinline__ int last(int w) const { return (r0 + bh - 1) * w + c0 + bw - 1; }
};

__device__ __forceinline__ Box weight_box(const MomState& st, int h, int w) {
    const float gg = st.g1 * st.g1 + st.g2 * st.g2;
    const float rc = kWeightCut * st.sw / (1.f - gg);
    const float hx = fminf(rc * sqrtf(1.f + gg + 2.f * st.g1) + 1.f, 4096.f);
    const float hy = fminf(rc * sqrtf(1.f + gg - 2.f * st.g1) + 1.f, 4096.f);
    const float xc = static_cast<float>(st.xi) + st.xf, yc = static_cast<float>(st.yi) + st.yf;
    Box b;
    b.c0 = max(0, static_cast<int>(floorf(xc - hx)));
    b.r0 = max(0, static_cast<int>(floorf(yc - hy)));
    const int c1 = min(w - 1, static_cast<int>(ceilf(xc + hx)));
    const int r1 = min(h - 1, static_cast<int>(ceilf(yc + hy)));
    // a centre outside the stamp (the iteration then stops) or a non-finite
    // state falls back to the whole stamp
    if (!(c1 >= b.c0 && r1 >= b.r0) || !(hx > 0.f && hy > 0.f)) {
        b.c0 = b.r0 = 0;
        b.bw = w;
        b.bh = h;
    } else {
        b.bw = c1 - b.c0 + 1;
        b.bh = r1 - b.r0 + 1;
    }
    return b;
}

// The pixels q = t, t + nt, ... of a box, row-major within it (the stamp
// index p grows with q, so a walk ends once p passes the box's last pixel;
// a thread with t beyond the box starts past it): their offsets
// (column - xr, row - yr) from the reference pixel and their index in the
// stamp of width w.  The offsets are integers below 2^24, exact in fp32, so
// stepping them with float adds gives the same values as converting the
// integer offsets, without a conversion per pixel.
struct BoxWalk {
    float u, v;
    int p;
    float du, dv, wrap, fbw;
    int dp, dwrap;
    __device__ __forceinline__ BoxWalk(int t, const Box& b, int w, int nt, int xr, int yr) {
        const int row = t / b.bw, col = t - row * b.bw;
        const int dr = nt / b.bw, dc = nt - dr * b.bw;
        u = static_cast<float>(b.c0 + col - xr);
        v = static_cast<float>(b.r0 + row - yr);
        p = (b.r0 + row) * w + b.c0 + col;
        du = static_cast<float>(dc);
        dv = static_cast<float>(dr);
        wrap = static_cast<float>(b.c0 + b.bw - xr);
        fbw = static_cast<float>(b.bw);
        dp = dr * w + dc;
        dwrap = w - b.bw;
    }
    __device__ __forceinline__ void next() {
        u += du;
        v += dv;
        p += dp;
        if (u >= wrap) {
            u -= fbw;
            v += 1.f;
            p += dwrap;
        }
    }
};

// One weighted pass: S0 = sum f W, S1 = sum f W theta, the three second and
// (FOURTH) five fourth moments of f W (f = pixel value).  Everything the
// centroid step (Eqs. 5-6) and the ellipticity step (Eqs. 8-9 with A5-A6,
// B7-B14) needs is a linear combination of these eleven sums.  The fourth
// moments only shape the step of Eq. 9 (through P^SH) and the matched weight's
// derivative, not the fixed point; a pass without them leaves acc[6..10] as
// they were (the last pass that summed them).
template <int NW, bool FOURTH>
__device__ __forceinline__ void moment_pass(const float* __restrict__ s, int w, const Box& bx,
                                            const Grp<NW>& g, const MomState& st,
                                            float (&acc)[11]) {
    const float gg = st.g1 * st.g1 + st.g2 * st.g2;
    const float A = 1.f + gg - 2.f * st.g1;
    const float B = 1.f + gg + 2.f * st.g1;
    const float G4 = 4.f * st.g2;
    const float cw = -kLog2e / (2.f * st.sw * st.sw);
    constexpr int N = FOURTH ? 11 : 6;
#pragma unroll
    for (int i = 0; i < N; ++i) acc[i] = 0.f;
    // centre relative to the reference pixel; rounding it to fp32 here costs
    // at most 2.4e-7 px, below the noise of these sums (the refinement passes
    // use exact offsets)
    const float cx = static_cast<float>(st.xi - st.xr) + st.xf;
    const float cy = static_cast<float>(st.yi - st.yr) + st.yf;
    // pixel offsets from the reference pixel, exact integers in fp32
    BoxWalk ow(g.t, bx, w, Grp<NW>::NT, st.xr, st.yr);
    const int plast = bx.last(w);   // the walk's index grows with each step
#pragma unroll 2
    while (ow.p <= plast) {
        const float t1 = ow.u - cx;
        const float t2 = ow.v - cy;
        const float I = s[ow.p];
        ow.next();
        const float t11 = t1 * t1, t22 = t2 * t2, t12 = t1 * t2;
        const float R2 = fmaf(A, t11, fmaf(B, t22, -G4 * t12));
        const float f = I * ex2(R2 * cw);
        acc[0] += f;
        acc[1] = fmaf(f, t1, acc[1]);
        acc[2] = fmaf(f, t2, acc[2]);
        acc[3] = fmaf(f, t11, acc[3]);
        acc[4] = fmaf(f, t12, acc[4]);
        acc[5] = fmaf(f, t22, acc[5]);
        if constexpr (FOURTH) {
            const float f11 = f * t11, f22 = f * t22;
            acc[6] = fmaf(f11, t11, acc[6]);    // theta1^4
            acc[7] = fmaf(f11, t12, acc[7]);    // theta1^3 theta2
            acc[8] = fmaf(f11, t22, acc[8]);    // theta1^2 theta2^2
            acc[9] = fmaf(f22, t12, acc[9]);    // theta1 theta2^3
            acc[10] = fmaf(f22, t22, acc[10]);  // theta2^4
        }
    }
    if constexpr (FOURTH) {
        g.allsum(acc);
    } else {
        float a6[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) a6[i] = acc[i];
        g.allsum(a6);
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i] = a6[i];
    }
}

struct MomStep {
    float dx, dy, dg1, dg2, sw_new;
    bool ok;
};

struct Pol {
    float P11, P12, P21, P22;
};

__device__ __noinline__ Pol shear_polarizability(float Q11, float Q12, float Q22, float F40, float F31,
                                                 float F22, float F13, float F04, float g1, float g2,
                                                 float sw, float e1, float e2);

// The centroid step <x>/N = k dx (Eqs. 5-6) and the ellipticity step
// dg = (1-|g_w|^2) (P^SH)^-1 (e^obs - e_w) (Eq. 9) with
// P^SH = X^SH + dX^SH - e (e^SH + de^SH)^T (Eq. 8, A5, A6, B7, B8), evaluated
// from the eleven weighted moments.  W' = dW/dR^2 = -c W with c = 1/(2 s_w^2).
__device__ __forceinline__ MomStep moment_step(const float (&m)[11], const MomState& st,
                                               float k_gain, bool ellip, bool matched) {
    MomStep r;
    r.ok = false;
    r.dx = r.dy = r.dg1 = r.dg2 = 0.f;
    r.sw_new = st.sw;
    const float S0 = m[0];
    const float Q11 = m[3], Q12 = m[4], Q22 = m[5];
    const float g1 = st.g1, g2 = st.g2;
    const float gg = g1 * g1 + g2 * g2;
    const float A = 1.f + gg - 2.f * g1, B = 1.f + gg + 2.f * g1;
    if (!(S0 > 0.f)) return r;
    const float c = 1.f / (2.f * st.sw * st.sw);
    // Eqs. 5-6 with the fixed gain k (k_gain, or 0.75 where the determined
    // gain below is not usable)
    const float kf = k_gain > 0.f ? k_gain : 0.75f;
    const float ik = 1.f / (kf * S0);
    r.dx = m[1] * ik;
    r.dy = m[2] * ik;
    if (k_gain <= 0.f) {
        // k determined from the current moments: the derivative of
        // (sum I W theta_1, sum I W theta_2) with respect to the centre, which
        // for a Gaussian profile is k = s_w^2 / (s^2 + s_w^2) (Sec. 2).  It is
        // used near the fixed point only (fixed-gain step below 0.25 px, where
        // the linearisation holds), when the Jacobian is positive definite and
        // the gain it implies, |M1| / (S0 |step|), lies in [0.15, 1.5], and
        // the weight is wider than 0.6 px: far from the fixed point a noisy
        // first moment with a small gain jumps out of the stamp, and a weight
        // about as narrow as a pixel (sigma_w clamped at 0.5) makes the
        // moments pixelated and the derivative meaningless.
        const float J11 = 2.f * c * (A * Q11 - 2.f * g2 * Q12) - S0;
        const float J12 = 2.f * c * (B * Q12 - 2.f * g2 * Q11);
        const float J21 = 2.f * c * (A * Q12 - 2.f * g2 * Q22);
        const float J22 = 2.f * c * (B * Q22 - 2.f * g2 * Q12) - S0;
        const float dj = J11 * J22 - J12 * J21;
        const float idj = 1.f / dj;
        const float nx = -(J22 * m[1] - J12 * m[2]) * idj;
        const float ny = -(-J21 * m[1] + J11 * m[2]) * idj;
        // |M1| against S0 |n| compared squared: [0.15, 1.5] -> [0.0225, 2.25]
        const float num2 = m[1] * m[1] + m[2] * m[2];
        const float den2 = S0 * S0 * (nx * nx + ny * ny);
        const bool near = fmaxf(fabsf(r.dx), fabsf(r.dy)) < 0.25f && st.sw > 0.6f;
        if (near && dj > 0.f && isfinite(nx) && isfinite(ny) &&
            (den2 == 0.f || (num2 >= 0.0225f * den2 && num2 <= 2.25f * den2))) {
            r.dx = nx;
            r.dy = ny;
        }
    }
    if (matched) {
        const float SR2 = A * Q11 + B * Q22 - 4.f * g2 * Q12;      // sum f W R^2
        r.sw_new = SR2 > 0.f ? sqrtf(SR2 / S0) : 0.f;
        // The matched-weight rule s_w^2 = S(s_w) = sum f W R^2 / sum f W contracts
        // slowly for cuspy profiles; near its fixed point take a Newton step on
        // s_w^2 - S(s_w) = 0 instead, with dS/ds_w = (<R^4> - <R^2>^2) / s_w^3
        // (<.> the f W - weighted means; sum f W R^4 from the fourth moments).
        // The fixed point is the same.
        const float G4 = 4.f * g2;
        const float SR4 = A * A * m[6] + B * B * m[10] + (G4 * G4 + 2.f * A * B) * m[8] -
                          2.f * A * G4 * m[7] - 2.f * B * G4 * m[9];
        const float sw = st.sw, S = SR2 / S0;
        const float dS = (SR4 / S0 - S * S) / (sw * sw * sw);
        const float dF = 2.f * sw - dS;
        const float sn = sw - (sw * sw - S) / dF;
        if (fabsf(r.sw_new - sw) < 0.2f * sw && dF > 0.1f * sw && sn > 0.5f * sw && sn < 1.5f * sw &&
            isfinite(sn))
            r.sw_new = sn;
    }
    if (!ellip) {
        r.ok = isfinite(r.dx) && isfinite(r.dy);
        return r;
    }
    const float T = Q11 + Q22;
    if (!(T > 0.f)) return r;
    const float iT = 1.f / T;
    const float e1 = (Q11 - Q22) * iT, e2 = 2.f * Q12 * iT;
    const Pol P = shear_polarizability(Q11, Q12, Q22, m[6], m[7], m[8], m[9], m[10], g1, g2, st.sw, e1, e2);
    const float det = P.P11 * P.P22 - P.P12 * P.P21;
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return r;
    const float ew = 2.f / (1.f + gg);
    const float r1 = e1 - ew * g1, r2 = e2 - ew * g2;
    const float sc = (1.f - gg) / det;
    r.dg1 = sc * (P.P22 * r1 - P.P12 * r2);
    r.dg2 = sc * (-P.P21 * r1 + P.P11 * r2);
    r.ok = isfinite(r.dg1) && isfinite(r.dg2) && isfinite(r.dx) && isfinite(r.dy);
    return r;
}

// P^SH = X^SH + dX^SH - e (e^SH + de^SH)^T (Eq. 8 with A5, A6, B7, B8) from the
// second and fourth weighted moments; W' = dW/dR^2 = -c W with
// c = 1/(2 s_w^2).  Kept out of line: it is called once per pass from two
// places, and the moment kernel's code size (instruction fetch) matters more
// than a call; arguments and result travel in registers.
__device__ __noinline__ Pol shear_polarizability(float Q11, float Q12, float Q22, float F40, float F31,
                                                 float F22, float F13, float F04, float g1, float g2,
                                                 float sw, float e1, float e2) {
    const float gg = g1 * g1 + g2 * g2;
    const float A = 1.f + gg - 2.f * g1, B = 1.f + gg + 2.f * g1;
    const float T = Q11 + Q22;
    const float iT = 1.f / T;
    const float c = 1.f / (2.f * sw * sw);
    const float ApB = A + B, AmB = A - B;
    const float F31m13 = F31 - F13, F31p13 = F31 + F13;
    // Appendix A: sum f W chi_a psi_b and sum f W theta^2 psi_b
    const float c1p1 = A * F40 - ApB * F22 + B * F04;
    const float c1p2 = ApB * F31m13 - 2.f * g2 * (F40 - F04);
    const float c2p1 = 2.f * (A * F31 - B * F13);
    const float c2p2 = 2.f * ApB * F22 - 4.f * g2 * F31p13;
    const float t2p1 = A * F40 + AmB * F22 - B * F04;
    const float t2p2 = ApB * F31p13 - 2.f * g2 * (F40 + 2.f * F22 + F04);
    float X11 = 2.f - 2.f * c * c1p1 * iT;
    float X12 = -2.f * c * c1p2 * iT;
    float X21 = -2.f * c * c2p1 * iT;
    float X22 = 2.f - 2.f * c * c2p2 * iT;
    float eS1 = 2.f * e1 - 2.f * c * t2p1 * iT;
    float eS2 = 2.f * e2 - 2.f * c * t2p2 * iT;
    // Appendix B: sum f P_1 ... P_6
    const float D = Q11 - Q22;
    const float P1 = 4.f * D - 2.f * c * (A * F40 - AmB * F22 - B * F04 - 4.f * g2 * F31m13);
    const float P2 = 4.f * Q12 - 2.f * c * (AmB * F31m13 + 2.f * g2 * (F40 - 2.f * F22 + F04));
    const float P3 = 8.f * Q12 - 4.f * c * (A * F31 + B * F13 - 4.f * g2 * F22);
    const float P4 = -2.f * D - 4.f * c * (AmB * F22 + 2.f * g2 * F31m13);
    const float P5 = 4.f * T - 2.f * c * (A * F40 + ApB * F22 + B * F04 - 4.f * g2 * F31p13);
    const float P6 = -2.f * c * (AmB * F31p13 + 2.f * g2 * (F40 - F04));
    X11 += (-g1 * P1 - g2 * P2) * iT;
    X12 += (g1 * P2 - g2 * P1) * iT;
    X21 += (-g1 * P3 - g2 * P4) * iT;
    X22 += (g1 * P4 - g2 * P3) * iT;
    eS1 += (-g1 * P5 - g2 * P6) * iT;
    eS2 += (g1 * P6 - g2 * P5) * iT;
    Pol P;
    P.P11 = X11 - e1 * eS1;
    P.P12 = X12 - e1 * eS2;
    P.P21 = X21 - e2 * eS1;
    P.P22 = X22 - e2 * eS2;
    return P;
}

// Final refinement of the fixed point: one pass with the pixel offsets theta
// (the fourth moments F, which only shape the step of Eq. 9 and the matched
// weight's derivative, come from the iteration's last pass, a step away)
// kept exactly as float pairs, the weight's exponent R^2 / (2 s_w^2) carried
// as a float pair (the rounding of every step of Eq. A1 kept), W to about one
// ulp (exp2_acc), and the zeroth, first and second moments accumulated in
// double-float with the rounding of each product kept; then one step from
// these sums: a Newton step for the centre (the derivative of the weighted
// first moments, i.e. k taken from the moments), the step of Eq. 9 for g and,
// for the matched weight, a Newton step for s_w.  The fp32 iteration stops
// within the noise of its own sums (~1e-6 px); this pass removes most of
// that noise.  The fixed point's accuracy is set by the weights' rounding:
// with an fp32 exponent (relative errors of ~2e-7 at two weight sizes) the
// centre moved by ~1e-7 px, which first-order chi^2 sensitivities of up to
// ~6e5 per px on bright stamps turn into 1e-5 of chi^2.  The sums run over
// the weight's box (weight_box).  Returns the largest move (pixels, g, and
// s_w relative), or -1 when no step was taken (singular sums, or a step
// larger than the iteration's own noise).
template <int NW>
__device__ float moment_refine(const float* __restrict__ s, int h, int w, const Grp<NW>& g,
                               bool ellip, bool matched, float sw_max, const float (&F)[5], MomState& st) {
    const float gg = st.g1 * st.g1 + st.g2 * st.g2;
    const float A = 1.f + gg - 2.f * st.g1;
    const float B = 1.f + gg + 2.f * st.g1;
    const float G4 = 4.f * st.g2;
    const float cw = -kLog2e / (2.f * st.sw * st.sw);
    float dh[6], dl[6], cx[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) dh[i] = dl[i] = cx[i] = 0.f;
    const Box bx = weight_box(st, h, w);
    BoxWalk ow(g.t, bx, w, Grp<NW>::NT, st.xi, st.yi);
    const int plast = bx.last(w);
#pragma unroll 1
    while (ow.p <= plast) {
        const int p = ow.p;
        const float k1 = ow.u, k2 = ow.v;
        // theta = k - x_f exactly as hi + lo (|k| >= |x_f| unless k = 0, where lo = 0)
        const float t1 = k1 - st.xf, t1l = -st.xf - (t1 - k1);
        const float t2 = k2 - st.yf, t2l = -st.yf - (t2 - k2);
        // theta_a theta_b as hi + lo: the rounding of the product and the first-order low parts
        const float p11 = t1 * t1, e11 = fmaf(t1, t1, -p11) + 2.f * t1 * t1l;
        const float p22 = t2 * t2, e22 = fmaf(t2, t2, -p22) + 2.f * t2 * t2l;
        const float p12 = t1 * t2, e12 = fmaf(t1, t2, -p12) + fmaf(t1, t2l, t1l * t2);
        // R^2 = A theta1^2 + B theta2^2 - 4 g2 theta1 theta2 (Eq. A1) as hi + lo
        const float ra = A * p11, rb = B * p22, rc = G4 * p12;
        const float s1 = ra + rb;
        const float s1e = (ra - (s1 - (s1 - ra))) + (rb - (s1 - ra));
        const float R2 = s1 - rc;
        const float R2e = (s1 - (R2 - (R2 - s1))) + (-rc - (R2 - s1));
        const float R2l = (fmaf(A, p11, -ra) + fmaf(B, p22, -rb) - fmaf(G4, p12, -rc)) + (s1e + R2e) +
                          fmaf(A, e11, fmaf(B, e22, -G4 * e12));
        const float x = R2 * cw;
        const float xl = fmaf(R2, cw, -x) + R2l * cw;
        const float Wh = exp2_acc(x);
        const float W = fmaf(Wh, xl * static_cast<float>(kLn2), Wh);
        const float I = s[p];
        const float f = I * W, fl = fmaf(I, W, -f);
        float q;
        df_add(dh[0], dl[0], f);
        cx[0] += fl;
        q = f * t1;
        df_add(dh[1], dl[1], q);
        cx[1] += fmaf(f, t1, -q) + fmaf(f, t1l, fl * t1);
        q = f * t2;
        df_add(dh[2], dl[2], q);
        cx[2] += fmaf(f, t2, -q) + fmaf(f, t2l, fl * t2);
        q = f * p11;
        df_add(dh[3], dl[3], q);
        cx[3] += fmaf(f, p11, -q) + fmaf(f, e11, fl * p11);
        q = f * p12;
        df_add(dh[4], dl[4], q);
        cx[4] += fmaf(f, p12, -q) + fmaf(f, e12, fl * p12);
        q = f * p22;
        df_add(dh[5], dl[5], q);
        cx[5] += fmaf(f, p22, -q) + fmaf(f, e22, fl * p22);
        ow.next();
    }
    g.allsum_df(dh, dl);
    g.allsum(cx);
    // The first moments vanish at the fixed point; once accumulated exactly
    // they are small numbers that fp32 carries to full relative precision.
    const float M0 = dh[0] + (dl[0] + cx[0]);
    const float M1x = dh[1] + (dl[1] + cx[1]);
    const float M1y = dh[2] + (dl[2] + cx[2]);
    const float Q11 = dh[3] + (dl[3] + cx[3]);
    const float Q12 = dh[4] + (dl[4] + cx[4]);
    const float Q22 = dh[5] + (dl[5] + cx[5]);
    if (!(M0 > 0.f) || !(Q11 + Q22 > 0.f)) return -1.f;
    const float c = 1.f / (2.f * st.sw * st.sw);
    const float g1 = st.g1, g2 = st.g2;
    const float J11 = 2.f * c * (A * Q11 - 2.f * g2 * Q12) - M0;
    const float J12 = 2.f * c * (B * Q12 - 2.f * g2 * Q11);
    const float J21 = 2.f * c * (A * Q12 - 2.f * g2 * Q22);
    const float J22 = 2.f * c * (B * Q22 - 2.f * g2 * Q12) - M0;
    const float dj = J11 * J22 - J12 * J21;
    if (!(dj > 0.f)) return -1.f;
    const float dx = -(J22 * M1x - J12 * M1y) / dj;
    const float dy = -(-J21 * M1x + J11 * M1y) / dj;
    // the second moments as doubles (a few operations per stamp): the
    // residuals below cancel at the fixed point
    const double M0d = static_cast<double>(dh[0]) + (static_cast<double>(dl[0]) + cx[0]);
    const double Q11d = static_cast<double>(dh[3]) + (static_cast<double>(dl[3]) + cx[3]);
    const double Q12d = static_cast<double>(dh[4]) + (static_cast<double>(dl[4]) + cx[4]);
    const double Q22d = static_cast<double>(dh[5]) + (static_cast<double>(dl[5]) + cx[5]);
    float dg1 = 0.f, dg2 = 0.f;
    if (ellip) {
        // e - e_w = [ (Q11 - Q22, 2 Q12) (1 + |g|^2) - 2 g T ] / (T (1 + |g|^2)): the
        // bracket cancels at the fixed point, so it is formed in fp64 before the
        // fp32 division.
        const double Td = Q11d + Q22d;
        const double opg = 1.0 + static_cast<double>(g1) * g1 + static_cast<double>(g2) * g2;
        const float n1 = static_cast<float>((Q11d - Q22d) * opg - 2.0 * g1 * Td);
        const float n2 = static_cast<float>(2.0 * Q12d * opg - 2.0 * g2 * Td);
        const float T = Q11 + Q22;
        const float den = T * (1.f + gg);
        const float r1 = n1 / den, r2 = n2 / den;
        const Pol P = shear_polarizability(Q11, Q12, Q22, F[0], F[1], F[2], F[3], F[4], g1, g2, st.sw,
                                           (Q11 - Q22) / T, 2.f * Q12 / T);
        const float P11 = P.P11, P12 = P.P12, P21 = P.P21, P22 = P.P22;
        const float det = P11 * P22 - P12 * P21;
        if (!(fabsf(det) > 0.f) || !isfinite(det)) return -1.f;
        const float sc = (1.f - gg) / det;
        dg1 = sc * (P22 * r1 - P12 * r2);
        dg2 = sc * (-P21 * r1 + P11 * r2);
    }
    float ds = 0.f;
    if (matched && st.sw > 0.5f && st.sw < sw_max) {
        // Newton on s_w^2 - sum f W R^2 / sum f W = 0 (the matched weight), the
        // residual formed in fp64; a step that would leave the clamp interval
        // is not taken (the iteration's clamped s_w stays)
        const double sw = st.sw;
        const double SR2 = static_cast<double>(A) * Q11d + static_cast<double>(B) * Q22d -
                           static_cast<double>(G4) * Q12d;
        const float res = static_cast<float>(sw * sw - SR2 / M0d);
        const float S = static_cast<float>(SR2 / M0d);
        const float SR4 = A * A * F[0] + B * B * F[4] + (G4 * G4 + 2.f * A * B) * F[2] -
                          2.f * A * G4 * F[1] - 2.f * B * G4 * F[3];
        const float dS = (SR4 / M0 - S * S) / (st.sw * st.sw * st.sw);
        const float dF = 2.f * st.sw - dS;
        ds = dF > 0.f ? -res / dF : 0.f;
        if (!(st.sw + ds > 0.5f && st.sw + ds < sw_max) || !isfinite(ds)) ds = 0.f;
    }
    // a refinement moves the point by at most the iteration's own noise
    if (!(fabsf(dx) <= 1e-3f && fabsf(dy) <= 1e-3f && fabsf(dg1) <= 1e-3f && fabsf(dg2) <= 1e-3f &&
          fabsf(ds) <= 1e-3f * st.sw))
        return -1.f;
    st.xf += dx;
    st.yf += dy;
    st.g1 += dg1;
    st.g2 += dg2;
    st.sw += ds;
    return fmaxf(fmaxf(fmaxf(fabsf(dx), fabsf(dy)), fmaxf(fabsf(dg1), fabsf(dg2))), fabsf(ds) / st.sw);
}

constexpr float kMomRefineSkip = 1e-7f;
constexpr int kMomRefineMax = 4;   // refinement passes at most (matched weight; else one fewer)

// Iterate to the stop rule.  Returns the number of passes; sets status bits.
template <int NW>
__device__ int moment_iterate(const float* s, int h, int w, int npix, const Grp<NW>& g,
                              const DevOpts& o, bool ellip, MomState& st, uint32_t& status) {
    st.xr = st.xi;
    st.yr = st.yi;
    const float sw_max = 0.5f * static_cast<float>(h < w ? h : w);
    float prev = 0.f;   // size of the previous step, for the contraction estimate
    float F4[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // the last pass's fourth moments
    // with the determined gain (k_gain = 0): a centre step that does not shrink
    // switches the rest of the iteration to the fixed gain
    float k_use = o.k_gain, prev_c = 0.f;
    const float inv_tol_pos = 1.f / o.tol_pos, inv_tol_g = 1.f / o.tol_g, inv_tol_sig = 1.f / o.tol_sig;
    int it;
    float m[11];
    // the fourth moments are summed while the ellipticity (or the matched
    // weight size) still moves by more than 1e-3; later passes reuse them
    bool fourth = true;
    for (it = 1; it <= o.max_iter_mom; ++it) {
        const Box bx = weight_box(st, h, w);
        if (fourth)
            moment_pass<NW, true>(s, w, bx, g, st, m);
        else
            moment_pass<NW, false>(s, w, bx, g, st, m);
#pragma unroll
        for (int i = 0; i < 5; ++i) F4[i] = m[6 + i];
        const MomStep d = moment_step(m, st, k_use, ellip, o.sigw_mode == 0);
        if (k_use <= 0.f) {
            const float dc = fmaxf(fabsf(d.dx), fabsf(d.dy));
            if (it > 2 && dc >= prev_c) k_use = 0.75f;
            prev_c = dc;
        }
        if (!d.ok) {
            status |= FSE_ST_MOM_FAILED;
            break;
        }
        st.xf += d.dx;
        st.yf += d.dy;
        if (fabsf(st.xf) > 0.5f) {
            const float rr = rintf(st.xf);
            st.xi += static_cast<int>(rr);
            st.xf -= rr;
        }
        if (fabsf(st.yf) > 0.5f) {
            const float rr = rintf(st.yf);
            st.yi += static_cast<int>(rr);
            st.yf -= rr;
        }
        if (ellip) {
            // |g| < 1: a step past (1 + |g_w|)/2 is shortened radially to it
            const float cap = 0.5f * (1.f + sqrtf(st.g1 * st.g1 + st.g2 * st.g2));
            float n1 = st.g1 + d.dg1, n2 = st.g2 + d.dg2;
            const float nn2 = n1 * n1 + n2 * n2;
            if (nn2 > cap * cap) {
                const float f = cap * rsqrtf(nn2);
                n1 *= f;
                n2 *= f;
            }
            st.g1 = n1;
            st.g2 = n2;
        }
        fourth = it < 3 || fmaxf(fabsf(d.dg1), fabsf(d.dg2)) > 1e-3f ||
                 (o.sigw_mode == 0 && fabsf(d.sw_new - st.sw) > 1e-3f * st.sw);
        float dsig = 0.f;
        if (o.sigw_mode == 0) {
            float ns = d.sw_new;
            if (ns < 0.5f) { ns = 0.5f; status |= FSE_ST_SIGW_CLAMPED; }
            if (ns > sw_max) { ns = sw_max; status |= FSE_ST_SIGW_CLAMPED; }
            dsig = __fdividef(fabsf(ns - st.sw), st.sw);
            st.sw = ns;
        }
        const float xc = static_cast<float>(st.xi) + st.xf, yc = static_cast<float>(st.yi) + st.yf;
        if (st.g1 * st.g1 + st.g2 * st.g2 >= 0.95f * 0.95f || xc < -0.5f ||
            xc > static_cast<float>(w) - 0.5f || yc < -0.5f || yc > static_cast<float>(h) - 0.5f) {
            status |= FSE_ST_MOM_FAILED;
            break;
        }
        // Stop when the distance left to the fixed point is below the
        // tolerances.  For a slowly contracting iteration that distance is
        // estimated as |step| rho / (1 - rho) with rho = |step_k| / |step_k-1|;
        // steps below a quarter of the tolerances (where the fp32 sums' noise
        // makes rho meaningless) always stop.
        // (step sizes in units of the tolerances; the stop rule needs no
        // correctly rounded quotients)
        const float sz = fmaxf(fmaxf(fabsf(d.dx), fabsf(d.dy)) * inv_tol_pos,
                               fmaxf(fmaxf(fabsf(d.dg1), fabsf(d.dg2)) * inv_tol_g, dsig * inv_tol_sig));
        const float rho = prev > 0.f ? fminf(__fdividef(sz, prev), 0.95f) : 0.f;
        const float left = (sz > 0.25f && rho > 0.5f) ? __fdividef(sz * rho, 1.f - rho) : sz;
        prev = sz;
        if (left <= 1.f) {
            status |= FSE_ST_MOM_CONVERGED;
            break;
        }
    }
    if (it > o.max_iter_mom) {
        status |= FSE_ST_MOM_MAXITER;
        it = o.max_iter_mom;
    }
    // refinement steps: the first leaves about a tenth of its own step (the
    // centre, g and s_w steps are taken separately); another runs while the
    // last moved the point by more than kMomRefineSkip, up to kMomRefineMax
    // passes for the matched weight (whose s_w step couples to the others
    // most strongly, for weights of a pixel or less) and one fewer otherwise.
    // A step the refinement does not take (negative return) ends them.
    if (status & FSE_ST_MOM_CONVERGED) {
        // one call site: the pass is large code
        const int rmax = o.sigw_mode == 0 ? kMomRefineMax : kMomRefineMax - 1;
#pragma unroll 1
        for (int r = 0; r < rmax; ++r) {
            if (r == 1) status |= FSE_ST_MOM_REFINE2;
            const float moved = moment_refine(s, h, w, g, ellip, o.sigw_mode == 0, sw_max, F4, st);
            if (moved <= kMomRefineSkip) break;
        }
    }
    return it;
}

// ------------------------------------------------------------------ start-up
struct InitOut {
    int peak;        // brightest pixel (lowest index on ties)
    float r50;
    bool finite;
    bool fallback;   // stamp total <= 0
    bool overflow;   // the stamp needs more rings than the tile holds (not expected)
};

// ceil(sqrt(d2)) for an integer 0 <= d2 <= 2 * 127^2 (sides of at most
// FSE_MAX_SIDE = 128 pixels), with one MUFU operation and integer arithmetic:
// d2 becomes a float through the bits of 2^23 + d2 (exact below 2^23), and the
// root is rounded to the nearest integer k0 by adding 2^23 (whose ulp is 1).
// sqrt.approx.f32 is within about 2^-22 relative of the square root, under
// 1e-4 here, so k0 is the floor or the ceiling of the true root, and the
// comparison k0^2 < d2 turns either into the ceiling.
__device__ __forceinline__ int ring_of(int d2) {
    const float f = __int_as_float(0x4B000000 | d2) - 8388608.f;
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(f));
    const int k0 = __float_as_int(r + 8388608.f) - 0x4B000000;
    return k0 + (k0 * k0 < d2 ? 1 : 0);
}

// Brightest pixel, and the half-light radius r50 from the growth curve around
// it (Sec. 4.1): pixels are binned in rings of integer radius k (k-1 < d <= k)
// and the enclosed sum is tracked until it reaches half the stamp total; r50
// interpolates linearly in the ring that crosses.  Sums are exact 64-bit
// fixed point (pixel * 2^S), so the crossing ring does not depend on the
// summation order.  Each 64-bit value q is accumulated as three 32-bit
// pieces, q = q2 2^(2b) + q1 2^b + q0 with 0 <= q0, q1 < 2^b and
// b = 31 - ceil(log2 npix): no piece's sum over the stamp can leave 32 bits,
// so native 32-bit shared-memory atomics add them exactly.
template <int NW>
__device__ InitOut stamp_init(const float* s, int h, int w, int npix, const Grp<NW>& g,
                              unsigned* hist, int slots) {
    constexpr int NT = Grp<NW>::NT;
    const int lane = g.lane;
    InitOut o;
    float vmax = -INFINITY, amax = 0.f;
    int imax = 0x7fffffff;
    bool fin = true;
    for (int p = g.t; p < npix; p += NT) {
        const float v = s[p];
        fin = fin && isfinite(v);
        if (v > vmax) { vmax = v; imax = p; }
        amax = fmaxf(amax, fabsf(v));
    }
    o.finite = g.all(fin);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(kFull, vmax, off);
        const int oi = __shfl_xor_sync(kFull, imax, off);
        if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
        amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, off));
    }
    if (NW > 1) {
        // the same rule across the group's warps, in warp order
        g.sync();
        if (lane == 0) {
            g.red[g.wi * 32] = vmax;
            g.red[g.wi * 32 + 1] = __int_as_float(imax);
            g.red[g.wi * 32 + 2] = amax;
        }
        g.sync();
        vmax = g.red[0];
        imax = __float_as_int(g.red[1]);
        amax = g.red[2];
        for (int k = 1; k < NW; ++k) {
            const float ov = g.red[k * 32];
            const int oi = __float_as_int(g.red[k * 32 + 1]);
            if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
            amax = fmaxf(amax, g.red[k * 32 + 2]);
        }
    }
    o.peak = imax;
    o.fallback = false;
    o.overflow = false;
    o.r50 = static_cast<float>(kSqrt2Ln2);
    if (!o.finite) return o;
    const int pr = imax / w, pc = imax - (imax / w) * w;
    // fixed-point scale 2^S with amax * npix * 2^S < 2^62
    int e;
    frexpf(amax * static_cast<float>(npix), &e);
    int S = 62 - e;
    S = S > 100 ? 100 : (S < -100 ? -100 : S);
    const float fs = ldexpf(1.f, S);
    // the largest row and column distance from the brightest pixel to an edge
    const int dh = (h - 1 - pr > pr ? h - 1 - pr : pr), dw = (w - 1 - pc > pc ? w - 1 - pc : pc);
    const int kmax = static_cast<int>(ceilf(sqrtf(static_cast<float>(dh * dh + dw * dw)))) + 1;
    const int nb = kmax + 1;
    if (nb > slots) {   // the tile is sized for every stamp it may hold; kept as a guard
        o.overflow = true;
        return o;
    }
    unsigned* h0 = hist;
    unsigned* h1 = hist + nb;
    int* h2 = reinterpret_cast<int*>(hist + 2 * nb);
    for (int k = g.t; k < 3 * nb; k += NT) hist[k] = 0u;
    g.sync();
    const int b = 31 - (npix > 1 ? 32 - __clz(npix - 1) : 0);
    const unsigned mask = (1u << b) - 1u;
    // Each thread takes a block of Cb consecutive pixels, Cb odd: the threads
    // of a warp sit about Cb pixels apart (a row or more), mostly on
    // different rings, so the atomics of one instruction seldom meet on one
    // address, and their pixel loads fall in distinct banks.  The sums are
    // integers, so the order of the additions does not change them.
    {
        const int Cb = ((npix + NT - 1) / NT) | 1;
        const int b0 = g.t * Cb;
        const int pend = b0 + Cb < npix ? b0 + Cb : npix;
        int row = b0 / w, col = b0 - row * w;
        int di = row - pr, dj = col - pc;
        int d2 = di * di + dj * dj;
#pragma unroll 1
        for (int p = b0; p < pend; ++p) {
            const long long q = __float2ll_rn(s[p] * fs);
            const int k = ring_of(d2);
            atomicAdd(&h0[k], static_cast<unsigned>(q) & mask);
            atomicAdd(&h1[k], static_cast<unsigned>(static_cast<unsigned long long>(q) >> b) & mask);
            atomicAdd(&h2[k], static_cast<int>(q >> (2 * b)));
            // the next pixel: one column on, or the first of the next row
            d2 += 2 * dj + 1;
            ++dj;
            if (++col == w) {
                col = 0;
                ++di;
                dj = -pc;
                d2 = di * di + dj * dj;
            }
        }
    }
    g.sync();   // every ring of the histogram is complete (the scan reads them)
    // warp scan over the rings: lane owns rings [lane*ch, lane*ch + ch)
    const int ch = (nb + 31) / 32;
    const int k0 = lane * ch;
    long long own = 0;
    for (int k = k0; k < k0 + ch && k < nb; ++k)
        own += static_cast<long long>(h0[k]) + (static_cast<long long>(h1[k]) << b) +
               static_cast<long long>(h2[k]) * (1ll << (2 * b));
    long long incl = own;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long o2 = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += o2;
    }
    const long long tot = __shfl_sync(kFull, incl, 31);
    if (tot <= 0) {
        o.fallback = true;
        g.sync();   // the histogram's space is reused after this
        return o;
    }
    long long run = incl - own;     // enclosed sum before ring k0
    int kc = -1;
    long long prev = 0, cur = 0;
    for (int k = k0; k < k0 + ch && k < nb; ++k) {
        const long long nxt = run + static_cast<long long>(h0[k]) + (static_cast<long long>(h1[k]) << b) +
                              static_cast<long long>(h2[k]) * (1ll << (2 * b));
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
    kc = __shfl_sync(kFull, kc, src);
    prev = __shfl_sync(kFull, prev, src);
    cur = __shfl_sync(kFull, cur, src);
    if (kc <= 0) {
        o.r50 = kc == 0 ? 0.25f * static_cast<float>(tot) / static_cast<float>(cur)
                        : static_cast<float>(kSqrt2Ln2);
    } else {
        // (half - prev) / (cur - prev) with the differences taken exactly in integers
        o.r50 = static_cast<float>(kc - 1) + static_cast<float>(tot - 2 * prev) /
                                                 (2.f * static_cast<float>(cur - prev));
    }
    g.sync();   // the histogram's space is reused after this
    return o;
}

// ------------------------------------------------------------------ fit
// One pass of the profile over the stamp at (I0g, r_e, n).  With
// a = log2(r/r_e), u = 2^(a/n) = (r/r_e)^(1/n), E = exp(-b u), v = E u and the
// residual r = I0g E - I, the ten sums below give chi^2, the normal equations
// of (I0, r_e, n) and, after eliminating I0 at its closed form (Eq. 13), the
// reduced 2x2 problem in (r_e, n):
//   dm/dr_e = I0 b v / (n r_e),  dm/dn = I0 (b ln2 / n^2) v a - I0 b'(n) v.
// Pixel-integrated model (fse_opts.supersample = S > 1): a pixel's model and
// its derivatives are the means over the S x S sub-grid points
// (t1 + (a + 1/2)/S - 1/2, t2 + (c + 1/2)/S - 1/2) of the pixel.  Everything the
// fit sums is linear in those means, so the sums and the solves are those of
// the pixel-centre model with each per-pixel factor replaced by its mean.
struct SubGeom {
    float A, B, G4;    // R^2 = A t1^2 + B t2^2 - G4 t1 t2 (Eq. A1)
    int S;
    float invS, invS2;
};

__device__ __forceinline__ SubGeom sub_geom(const MomState& st, int S) {
    const float gg = st.g1 * st.g1 + st.g2 * st.g2;
    SubGeom q;
    q.A = 1.f + gg - 2.f * st.g1;
    q.B = 1.f + gg + 2.f * st.g1;
    q.G4 = 4.f * st.g2;
    q.S = S;
    q.invS = 1.f / static_cast<float>(S);
    q.invS2 = q.invS * q.invS;
    return q;
}

// 0.5 log2 R^2 of a pixel or sub-grid point; at R = 0 (the centre itself) a
// value whose exp2 is 0.  The hardware lg2 is used: its absolute error (about
// 2^-22 on the logarithm of the mantissa) is that of the fp32 value it is kept
// in for the radii of a stamp, and it enters the model only through
// u = exp2((0.5 log2 R^2 - c0) / n), as an absolute error of the exponent.
__device__ __forceinline__ float half_log2_r2(float R2) {
    return R2 > 0.f ? 0.5f * __log2f(R2) : -1000.f;
}

// a = log2(r / r_e) of one sub-grid point (r = R / (1 - |g|); c0 = log2 r_e + log2(1 - |g|)).
__device__ __forceinline__ float sub_a(const SubGeom& q, float t1, float t2, int a, int c, float c0) {
    const float u1 = t1 + (static_cast<float>(a) + 0.5f) * q.invS - 0.5f;
    const float u2 = t2 + (static_cast<float>(c) + 0.5f) * q.invS - 0.5f;
    const float R2 = fmaf(q.A, u1 * u1, fmaf(q.B, u2 * u2, -q.G4 * (u1 * u2)));
    return half_log2_r2(R2) - c0;
}

// Offsets of a pixel from the fixed centre.
__device__ __forceinline__ void pix_t(const PixelWalk& pw, const MomState& st, float* t1, float* t2) {
    *t1 = static_cast<float>(pw.col - st.xi) - st.xf;
    *t2 = static_cast<float>(pw.row - st.yi) - st.yf;
}

struct FitEval {
    float I0;       // Eq. 13 at (r_e, n)
    float chi2;     // Eq. 11 at that I0
    float g[2];     // J^T r of the reduced problem
    float H[3];     // J^T J of the reduced problem (00, 01, 11)
    float corr;     // (I0 - I0g)^2 sum E^2 / chi2: cancellation in chi2 when large
};

template <bool IVAR, int NW, bool SUP = false>
__device__ FitEval fit_eval(const float* __restrict__ s, const float* __restrict__ L,
                            const float* __restrict__ sq, int npix, const Grp<NW>& g, float I0g,
                            float re, float n, float lq, int w = 0, const MomState* st = nullptr,
                            int S = 1) {
    float b, db;
    bn_eval_f(n, &b, &db);
    const float inv_n = 1.f / n;
    const float nbl = -b * kLog2e;
    const float c0 = log2f(re) + lq;
    float acc[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = 0.f;
    SubGeom sg;
    if constexpr (SUP) sg = sub_geom(*st, S);
    PixelWalk pw(g.t, SUP ? w : 1, Grp<NW>::NT);
    // four pixels in flight: their exp2 chains overlap, which the fit launch's
    // 12 warps per SM do not hide alone (2% faster than two)
#pragma unroll 4
    for (int p = g.t; p < npix; p += Grp<NW>::NT) {
        float E, v = 0.f, va = 0.f, u = 0.f, a = 0.f;
        if constexpr (SUP) {
            float t1, t2;
            pix_t(pw, *st, &t1, &t2);
            pw.next();
            E = 0.f;
            for (int ic = 0; ic < sg.S; ++ic)
                for (int ia = 0; ia < sg.S; ++ia) {
                    const float as = sub_a(sg, t1, t2, ia, ic, c0);
                    const float us = ex2(as * inv_n);
                    const float es = ex2(us * nbl);
                    E += es;
                    v = fmaf(es, us, v);
                    va = fmaf(es * us, as, va);
                }
            E *= sg.invS2;
            v *= sg.invS2;
            va *= sg.invS2;
        } else {
            a = L[p] - c0;
            u = ex2(a * inv_n);
            E = ex2(u * nbl);
        }
        float r = fmaf(I0g, E, -s[p]);
        if (IVAR) {
            const float q = sq[p];
            E *= q;
            r *= q;
            if constexpr (SUP) {
                v *= q;
                va *= q;
            }
        }
        if constexpr (!SUP) {
            v = E * u;
            va = v * a;
        }
        acc[0] = fmaf(E, E, acc[0]);
        acc[1] = fmaf(E, v, acc[1]);
        acc[2] = fmaf(E, va, acc[2]);
        acc[3] = fmaf(v, v, acc[3]);
        acc[4] = fmaf(v, va, acc[4]);
        acc[5] = fmaf(va, va, acc[5]);
        acc[6] = fmaf(E, r, acc[6]);
        acc[7] = fmaf(v, r, acc[7]);
        acc[8] = fmaf(va, r, acc[8]);
        acc[9] = fmaf(r, r, acc[9]);
    }
    g.allsum(acc);
    FitEval f;
    const float sEE = acc[0], sEv = acc[1], sEva = acc[2], svv = acc[3], svva = acc[4],
                svaa = acc[5], sEr = acc[6], svr = acc[7], svar = acc[8], srr = acc[9];
    const float iE = 1.f / sEE;
    const float d = -sEr * iE;                  // I0* - I0g
    f.I0 = I0g + d;
    f.chi2 = fmaf(d, sEr, srr);                 // = sum (I0* E - I)^2
    f.corr = d * d * sEE / fmaxf(f.chi2, 1e-30f);
    const float k2 = f.I0 * b / (n * re);
    const float kA = f.I0 * b * static_cast<float>(kLn2) * inv_n * inv_n;
    const float kB = f.I0 * db;
    const float svr_s = fmaf(d, sEv, svr), svar_s = fmaf(d, sEva, svar);
    const float Cvv = svv - sEv * sEv * iE;
    const float Cvva = svva - sEv * sEva * iE;
    const float Cvaa = svaa - sEva * sEva * iE;
    f.g[0] = k2 * svr_s;
    f.g[1] = kA * svar_s - kB * svr_s;
    f.H[0] = k2 * k2 * Cvv;
    f.H[1] = k2 * (kA * Cvva - kB * Cvv);
    f.H[2] = kA * kA * Cvaa - 2.f * kA * kB * Cvva + kB * kB * Cvv;
    return f;
}

// Start: r_e from the weight size, n the candidate of {0.5, 1, 2, 4} with the
// lowest chi^2 at its closed-form I0 (chi^2 = sum I^2 - (sum I E)^2 / sum E^2).
template <bool IVAR, int NW, bool SUP = false>
__device__ void fit_start(const float* __restrict__ s, const float* __restrict__ L,
                          const float* __restrict__ sq, int npix, const Grp<NW>& g, float re0,
                          float lq, float* n0, float* I00, int w = 0, const MomState* st = nullptr,
                          int S = 1) {
    const float nc[4] = {0.5f, 1.f, 2.f, 4.f};
    float inv_n[4], nbl[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float b, db;
        bn_eval_f(nc[c], &b, &db);
        inv_n[c] = 1.f / nc[c];
        nbl[c] = -b * kLog2e;
    }
    const float c0 = log2f(re0) + lq;
    float acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = 0.f;
    SubGeom sg;
    if constexpr (SUP) sg = sub_geom(*st, S);
    PixelWalk pw(g.t, SUP ? w : 1, Grp<NW>::NT);
    for (int p = g.t; p < npix; p += Grp<NW>::NT) {
        float I = s[p];
        const float q = IVAR ? sq[p] : 1.f;
        if (IVAR) I *= q;
        acc[8] = fmaf(I, I, acc[8]);
        if constexpr (SUP) {
            float t1, t2;
            pix_t(pw, *st, &t1, &t2);
            pw.next();
            float Em[4] = {0.f, 0.f, 0.f, 0.f};
            for (int ic = 0; ic < sg.S; ++ic)
                for (int ia = 0; ia < sg.S; ++ia) {
                    const float as = sub_a(sg, t1, t2, ia, ic, c0);
#pragma unroll
                    for (int c = 0; c < 4; ++c) Em[c] += ex2(ex2(as * inv_n[c]) * nbl[c]);
                }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float E = Em[c] * sg.invS2;
                if (IVAR) E *= q;
                acc[2 * c] = fmaf(E, E, acc[2 * c]);
                acc[2 * c + 1] = fmaf(E, I, acc[2 * c + 1]);
            }
        } else {
            const float a = L[p] - c0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float E = ex2(ex2(a * inv_n[c]) * nbl[c]);
                if (IVAR) E *= q;
                acc[2 * c] = fmaf(E, E, acc[2 * c]);
                acc[2 * c + 1] = fmaf(E, I, acc[2 * c + 1]);
            }
        }
    }
    g.allsum(acc);
    int best = 0;
    float bc = INFINITY;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float sEE = acc[2 * c], sEI = acc[2 * c + 1];
        const float chi2 = acc[8] - sEI * sEI / sEE;
        if (sEE > 0.f && chi2 < bc) {
            bc = chi2;
            best = c;
        }
    }
    *n0 = nc[best];
    *I00 = acc[2 * best] > 0.f ? acc[2 * best + 1] / acc[2 * best] : 1.f;
}

// Refinement at the LM optimum: a pass with both exponentials to
// about one ulp (exp2_acc), the residual sums sum E r, sum v r, sum v a r and
// sum r^2 accumulated in double-float (the J^T J sums in fp32), then one Newton
// step of the reduced problem and chi^2 from its quadratic model.  The fp32 LM stops
// within the noise of its own sums; this pass removes most of that noise.
// A precise evaluation of the profiled problem at (r_e, n): chi^2 at I0*, the
// Newton step for (r_e, n) (Gauss-Newton where the full Hessian is not
// positive definite), and what a step predicts.
struct Precise {
    double chi2;      // exact chi^2 at (I0*, r_e, n)
    double chi2_step; // chi^2 the quadratic model predicts after the full step
    float I0;         // I0* (Eq. 13 at this point)
    float d0, d1;     // Newton step for r_e, n (valid when ok)
    float c0, c1;     // dI0 = c0 d0 + c1 d1 along a step (Eq. 13 to first order)
    bool ok;
};


// fp64 squared residual of one bright pixel (kept out of line: rarely taken).
struct BrightModel {
    double b, lnre, ln1g, A, B, G4, inv_n, I0;
};

__device__ __noinline__ double bright_r2(const BrightModel& bm, double t1, double t2, float pix,
                                         float q) {
    const double R2 = bm.A * t1 * t1 + bm.B * t2 * t2 - bm.G4 * t1 * t2;
    const double u = exp((0.5 * log(R2) - bm.ln1g - bm.lnre) * bm.inv_n);
    const double r = (bm.I0 * exp(-bm.b * u) - pix) * q;
    return r * r;
}

// The same for the pixel-integrated model: the mean over the S x S sub-grid.
__device__ __noinline__ double bright_r2_sub(const BrightModel& bm, double t1, double t2, float pix,
                                             float q, int S) {
    double m = 0.0;
    for (int c = 0; c < S; ++c)
        for (int a = 0; a < S; ++a) {
            const double u1 = t1 + (a + 0.5) / S - 0.5, u2 = t2 + (c + 0.5) / S - 0.5;
            const double R2 = bm.A * u1 * u1 + bm.B * u2 * u2 - bm.G4 * u1 * u2;
            const double u = exp((0.5 * log(R2) - bm.ln1g - bm.lnre) * bm.inv_n);
            m += exp(-bm.b * u);
        }
    const double r = (bm.I0 * m / (static_cast<double>(S) * S) - pix) * q;
    return r * r;
}

// The scalar part of a refinement pass in precision R, from the
// double-float sums of the pass: I0* and chi^2 at I0*, then the Newton system
// over (r_e, n) with I0 profiled out (Schur complement).
template <typename R>
__device__ Precise refine_tail(const float (&rh)[10], const float (&rl)[10], const float (&T)[4],
                               double chi2_rr, float I0g, float re_f, float n_f, float bf, float dbf,
                               float d2bf) {
    R S[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) S[i] = static_cast<R>(rh[i]) + static_cast<R>(rl[i]);
    const R sEE = S[0], sEv = S[1], sEva = S[2], svv = S[3], svva = S[4], svaa = S[5];
    const R sEr = S[6], svr = S[7], svar = S[8];
    const R re = re_f, n = n_f, b = bf, db = dbf, d2b = d2bf;
    const R inv_n = R(1) / n;
    const R ln2 = static_cast<R>(kLn2);
    Precise o;
    const R d = -sEr / sEE;
    const R I0 = static_cast<R>(I0g) + d;
    // chi^2 at I0*: sum r^2 + d sum E r, with sum r^2 kept as a float pair
    o.chi2 = chi2_rr + static_cast<double>(d) * static_cast<double>(sEr);
    o.I0 = static_cast<float>(I0);
    const R k2 = I0 * b / (n * re);
    const R kA = I0 * b * ln2 * inv_n * inv_n;
    const R kB = I0 * db;
    const R svr_s = svr + d * sEv, svar_s = svar + d * sEva;
    const R Cvv = svv - sEv * sEv / sEE;
    const R Cvva = svva - sEv * sEva / sEE;
    const R Cvaa = svaa - sEva * sEva / sEE;
    // gradient of chi^2/2 over (r_e, n) at I0*
    const R g0 = k2 * svr_s, g1 = kA * svar_s - kB * svr_s;
    // Gauss-Newton part of the reduced Hessian (J^T J with I0 profiled out)
    R H00 = k2 * k2 * Cvv, H01 = k2 * (kA * Cvva - kB * Cvv);
    R H11 = kA * kA * Cvaa - R(2) * kA * kB * Cvva + kB * kB * Cvv;
    // J^T J couplings of I0 with r_e and n
    R JI0 = k2 * sEv, JI1 = kA * sEva - kB * sEv;
    {
        // Newton: add sum r d^2 m.  With phi = b u and E = exp(-phi),
        // d^2 E = E (dphi_i dphi_j - d^2 phi_ij); the derivatives of u = (r/r_e)^(1/n)
        // give the six residual sums r E u {1, a, a^2} and r E u^2 {1, a, a^2}
        // (a = log2(r/r_e)).  Where the residuals are large, dropping this term
        // leaves a Gauss-Newton iteration that converges slowly or not at all.
        const R c = inv_n / re;
        const R in2 = inv_n * inv_n;
        const R T0 = T[0], T1r = T[1], T2r = T[2], T3 = T[3];
        const R Srr = b * c * c * (b * T1r - (R(1) + n) * svr);
        const R Srn = c * (-b * db * T1r + b * b * ln2 * in2 * T2r + db * svr - b * ln2 * in2 * svar -
                           b * inv_n * svr);
        const R Snn = db * db * T1r - R(2) * b * db * ln2 * in2 * T2r + b * b * ln2 * ln2 * in2 * in2 * T3 -
                      d2b * svr + R(2) * db * ln2 * in2 * svar - b * ln2 * ln2 * in2 * in2 * T0 -
                      R(2) * b * ln2 * in2 * inv_n * svar;
        // the I0 rows gain g/I0 (sum r dE), which also enters the Schur complement
        const R q0 = g0 / I0, q1 = g1 / I0;
        const R N00 = H00 + I0 * Srr - (R(2) * JI0 * q0 + q0 * q0) / sEE;
        const R N01 = H01 + I0 * Srn - (JI0 * q1 + JI1 * q0 + q0 * q1) / sEE;
        const R N11 = H11 + I0 * Snn - (R(2) * JI1 * q1 + q1 * q1) / sEE;
        // keep Gauss-Newton where the full Hessian is not positive definite
        if (N00 > R(0) && N00 * N11 - N01 * N01 > R(0) && isfinite(N00 * N11)) {
            H00 = N00;
            H01 = N01;
            H11 = N11;
            JI0 += q0;
            JI1 += q1;
        }
    }
    const R det = H00 * H11 - H01 * H01;
    const R d0 = (-H11 * g0 + H01 * g1) / det;
    const R d1 = (H01 * g0 - H00 * g1) / det;
    o.ok = det > R(0) && isfinite(det) && isfinite(o.chi2) && isfinite(d0) && isfinite(d1);
    o.d0 = static_cast<float>(d0);
    o.d1 = static_cast<float>(d1);
    o.c0 = static_cast<float>(-JI0 / sEE);
    o.c1 = static_cast<float>(-JI1 / sEE);
    o.chi2_step = o.chi2 + static_cast<double>(R(2) * (g0 * d0 + g1 * d1) + d0 * (H00 * d0 + H01 * d1) +
                                               d1 * (H01 * d0 + H11 * d1));
    return o;
}

template <bool IVAR, int NW, bool SUP = false>
__device__ Precise fit_refine(const float* __restrict__ s, const float* __restrict__ L,
                              const float* __restrict__ sq, int w, int npix, const Grp<NW>& g,
                              float I0g,
                              float re, float n, float lq, const MomState& st, int S = 1) {
    float bf, dbf;
    bn_eval_f(n, &bf, &dbf);
    const float inv_n = 1.f / n;
    const float nbl = -bf * kLog2e;
    const float c0 = log2f(re) + lq;
    // fp64 model constants for the bright pixels of the final pass; a model
    // value exceeds the threshold only if |I0| does (E <= 1)
    const bool check_bright = IVAR || fabsf(I0g) > kBrightSigma;
    BrightModel bm;
    if (check_bright) {
        double dbd;
        bn_eval(static_cast<double>(n), &bm.b, &dbd);
        bm.lnre = log(static_cast<double>(re));
        const double g1 = st.g1, g2 = st.g2, gg = g1 * g1 + g2 * g2;
        bm.ln1g = log(1.0 - sqrt(gg));
        bm.A = 1.0 + gg - 2.0 * g1;
        bm.B = 1.0 + gg + 2.0 * g1;
        bm.G4 = 4.0 * g2;
        bm.inv_n = 1.0 / static_cast<double>(n);
        bm.I0 = I0g;
    }
    float rh[10], rl[10], T[4];
#pragma unroll
    for (int i = 0; i < 10; ++i) rh[i] = rl[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) T[i] = 0.f;
    PixelWalk pw(g.t, w, Grp<NW>::NT);
    if constexpr (SUP) {
        // the pixel-integrated model: every factor below is a mean over the sub-grid
        const SubGeom sg = sub_geom(st, S);
        for (int p = g.t; p < npix; p += Grp<NW>::NT) {
            float t1, t2;
            pix_t(pw, st, &t1, &t2);
            float E = 0.f, v = 0.f, va = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
            for (int ic = 0; ic < sg.S; ++ic)
                for (int ia = 0; ia < sg.S; ++ia) {
                    const float as = sub_a(sg, t1, t2, ia, ic, c0);
                    const float us = exp2_acc(as * inv_n);
                    const float es = exp2_acc(us * nbl);
                    const float eu = es * us, eua = eu * as, euu = eu * us;
                    E += es;
                    v += eu;
                    va += eua;
                    m0 = fmaf(eua, as, m0);        // E u a^2
                    m1 += euu;                     // E u^2
                    m2 = fmaf(euu, as, m2);        // E u^2 a
                    m3 = fmaf(euu * as, as, m3);   // E u^2 a^2
                }
            E *= sg.invS2;
            v *= sg.invS2;
            va *= sg.invS2;
            m0 *= sg.invS2;
            m1 *= sg.invS2;
            m2 *= sg.invS2;
            m3 *= sg.invS2;
            float r = fmaf(I0g, E, -s[p]);
            float rr_hi = 0.f, rr_lo = 0.f;
            bool bright = false;
            const float q = IVAR ? sq[p] : 1.f;
            if (check_bright && fabsf(I0g * E) * q > kBrightSigma) {
                const double rrd = bright_r2_sub(bm, static_cast<double>(pw.col - st.xi) - st.xf,
                                                 static_cast<double>(pw.row - st.yi) - st.yf, s[p], q, sg.S);
                rr_hi = static_cast<float>(rrd);
                rr_lo = static_cast<float>(rrd - rr_hi);
                bright = true;
            }
            pw.next();
            if (IVAR) {
                E *= q;
                r *= q;
                v *= q;
                va *= q;
                m0 *= q;
                m1 *= q;
                m2 *= q;
                m3 *= q;
            }
            rh[0] = fmaf(E, E, rh[0]);
            rh[1] = fmaf(E, v, rh[1]);
            rh[2] = fmaf(E, va, rh[2]);
            rh[3] = fmaf(v, v, rh[3]);
            rh[4] = fmaf(v, va, rh[4]);
            rh[5] = fmaf(va, va, rh[5]);
            df_add(rh[6], rl[6], E * r);
            df_add(rh[7], rl[7], v * r);
            df_add(rh[8], rl[8], va * r);
            T[0] = fmaf(r, m0, T[0]);
            T[1] = fmaf(r, m1, T[1]);
            T[2] = fmaf(r, m2, T[2]);
            T[3] = fmaf(r, m3, T[3]);
            if (bright) {
                df_add(rh[9], rl[9], rr_hi);
                rl[9] += rr_lo;
            } else {
                df_add(rh[9], rl[9], r * r);
            }
        }
    } else
    for (int p = g.t; p < npix; p += Grp<NW>::NT) {
        const float a = L[p] - c0;
        const float u = exp2_acc(a * inv_n);
        float E = exp2_acc(u * nbl);
        float r = fmaf(I0g, E, -s[p]);
        float rr_hi = 0.f, rr_lo = 0.f;
        bool bright = false;
        if (check_bright) {
            const float q = IVAR ? sq[p] : 1.f;
            if (fabsf(I0g * E) * q > kBrightSigma) {
                const double rrd = bright_r2(bm, static_cast<double>(pw.col - st.xi) - st.xf,
                                             static_cast<double>(pw.row - st.yi) - st.yf, s[p], q);
                rr_hi = static_cast<float>(rrd);
                rr_lo = static_cast<float>(rrd - rr_hi);
                bright = true;
            }
            pw.next();
        }
        if (IVAR) {
            const float q = sq[p];
            E *= q;
            r *= q;
        }
        const float v = E * u, va = v * a;
        const float vr = v * r, var = va * r;
        // J^T J (the first six sums) only shapes the Newton step: fp32.  The
        // gradient sums and chi^2, which cancel or must hold 1e-7 at the
        // optimum, are double-float.
        rh[0] = fmaf(E, E, rh[0]);
        rh[1] = fmaf(E, v, rh[1]);
        rh[2] = fmaf(E, va, rh[2]);
        rh[3] = fmaf(v, v, rh[3]);
        rh[4] = fmaf(v, va, rh[4]);
        rh[5] = fmaf(va, va, rh[5]);
        df_add(rh[6], rl[6], E * r);
        df_add(rh[7], rl[7], vr);
        df_add(rh[8], rl[8], var);
        // residual-weighted second-derivative sums of the model (Newton term)
        T[0] = fmaf(var, a, T[0]);       // r E u a^2
        T[1] = fmaf(vr, u, T[1]);        // r E u^2
        T[2] = fmaf(var, u, T[2]);       // r E u^2 a
        T[3] = fmaf(var * u, a, T[3]);   // r E u^2 a^2
        if (bright) {
            df_add(rh[9], rl[9], rr_hi);
            rl[9] += rr_lo;
        } else {
            df_add(rh[9], rl[9], r * r);
        }
    }
    g.allsum_df(rh, rl);
    g.allsum(T);
    // The sums are exact to about 1e-14 relative; the quantities that vanish at
    // the optimum (the gradient) are formed from them only after the
    // cancellation has happened inside the double-float sums.
    const double chi2_rr = static_cast<double>(rh[9]) + rl[9];
    return refine_tail<float>(rh, rl, T, chi2_rr, I0g, re, n, bf, dbf, bn_d2_f(n));
}

constexpr float kFitRefineSkip = 1e-4f;   // a Newton step below this ends the refinement
constexpr float kFitRefineCap = 0.2f;     // largest relative step of one refinement pass
constexpr float kFitRefineTrusted = 1e-2f; // steps up to this are taken without a chi^2 test
constexpr int kFitRefineMax = 16;         // refinement passes at most

struct FitOut {
    float I0, re, n, flux;
    double chi2;
    int iters;
};

// Levenberg-Marquardt over theta = (r_e, n) with I0 at its closed form after
// every pass; damping by the gain ratio rho (Nielsen 1999).
template <bool IVAR, int NW, bool SUP = false>
__device__ FitOut sersic_fit(const float* s, float* L, const float* sq, int h, int w, int npix,
                             const Grp<NW>& g, const DevOpts& o, const MomState& st,
                             uint32_t& status) {
    // per-pixel 0.5 log2 R^2 about the fixed centre with the fixed ellipticity
    // (the pixel-integrated model evaluates its sub-grid points as it goes)
    const float g1 = st.g1, g2 = st.g2;
    const float gg = g1 * g1 + g2 * g2;
    const float A = 1.f + gg - 2.f * g1, B = 1.f + gg + 2.f * g1, G4 = 4.f * g2;
    const int S = SUP ? o.supersample : 1;
    if constexpr (!SUP) {
        PixelWalk pw(g.t, w, Grp<NW>::NT);
        for (int p = g.t; p < npix; p += Grp<NW>::NT) {
            const float t1 = static_cast<float>(pw.col - st.xi) - st.xf;
            const float t2 = static_cast<float>(pw.row - st.yi) - st.yf;
            const float R2 = fmaf(A, t1 * t1, fmaf(B, t2 * t2, -G4 * (t1 * t2)));
            L[p] = half_log2_r2(R2);
            pw.next();
        }
        g.sync();
    }
    const float gabs = sqrtf(gg);
    const float lq = log2f(1.f - gabs);          // log2 r = 0.5 log2 R^2 - log2(1 - |g|)
    const float re_max = o.re_max_frac * static_cast<float>(h > w ? h : w);
    const float re_min = o.re_min, n_min = o.n_min, n_max = o.n_max;
    float re = static_cast<float>(kSqrt2Ln2) * st.sw / (1.f - gabs);
    re = re < re_min ? re_min : (re > re_max ? re_max : re);
    float n, I0g;
    fit_start<IVAR, NW, SUP>(s, L, sq, npix, g, re, lq, &n, &I0g, w, &st, S);
    // One evaluation site: every pass of the profile goes through the single
    // fit_eval call at the top of this loop (first the start, then each trial
    // step, and a repeat at I0* when the amplitude jumped).
    FitEval cur;
    cur.chi2 = INFINITY;
    bool have_cur = false, retried = false, converged = false, finite0 = true;
    float I0t = I0g, ret = re, nt = n, pred = 0.f;
    float lambda = o.lm_lambda0, nu = 2.f;
    int evals = 0, band_accepts = 0, it = 0;
#pragma unroll 1
    for (;;) {
        const FitEval ev = fit_eval<IVAR, NW, SUP>(s, L, sq, npix, g, I0t, ret, nt, lq, w, &st, S);
        ++evals;
        if (ev.corr > 0.5f && !retried) {
            // the amplitude moved so far that chi^2 lost precision: evaluate again at I0*
            I0t = ev.I0;
            retried = true;
            continue;
        }
        retried = false;
        if (!have_cur) {
            cur = ev;
            have_cur = true;
            finite0 = isfinite(cur.chi2) && isfinite(cur.g[0]) && isfinite(cur.g[1]) &&
                      isfinite(cur.H[0]) && isfinite(cur.H[1]) && isfinite(cur.H[2]);
            if (!finite0) {
                status |= FSE_ST_FIT_SINGULAR;
                break;
            }
        } else {
            // A step whose predicted decrease is below the resolution of the fp32
            // chi^2 is accepted when chi^2 stays within that resolution (at most a
            // few times), so that the iteration reaches the zero of the gradient
            // instead of stalling on rejections it cannot resolve.
            const float band = 1e-6f * cur.chi2;
            const bool better = ev.chi2 < cur.chi2;
            const bool in_band = pred <= band && ev.chi2 <= cur.chi2 + band && band_accepts < 4;
            if (better || in_band) {
                if (!better) ++band_accepts;
                const float rho = pred > 0.f ? (cur.chi2 - ev.chi2) / pred : 1.f;
                const float t = 2.f * rho - 1.f;
                lambda *= fmaxf(1.f / 3.f, 1.f - t * t * t);
                nu = 2.f;
                re = ret;
                n = nt;
                cur = ev;
            } else {
                lambda *= nu;
                nu *= 2.f;
                if (lambda > 1e15f) {
                    converged = true;
                    break;
                }
            }
        }
        if (++it > o.max_iter_fit) break;
        const float M00 = cur.H[0] * (1.f + lambda), M11 = cur.H[2] * (1.f + lambda);
        const float M01 = cur.H[1];
        const float det = M00 * M11 - M01 * M01;
        if (!(det > 0.f) || !isfinite(det)) {
            status |= FSE_ST_FIT_SINGULAR;
            break;
        }
        const float idet = 1.f / det;
        const float d0 = (-M11 * cur.g[0] + M01 * cur.g[1]) * idet;
        const float d1 = (M01 * cur.g[0] - M00 * cur.g[1]) * idet;
        float qre = re + d0, qn = n + d1;
        qre = qre < re_min ? re_min : (qre > re_max ? re_max : qre);
        qn = qn < n_min ? n_min : (qn > n_max ? n_max : qn);
        const float s0 = qre - re, s1 = qn - n;
        const float step = fmaxf(fabsf(s0) / re, fabsf(s1) / n);
        if (step <= o.tol_fit) {
            converged = true;
            break;
        }
        pred = -(2.f * (cur.g[0] * s0 + cur.g[1] * s1) + s0 * (cur.H[0] * s0 + cur.H[1] * s1) +
                 s1 * (cur.H[1] * s0 + cur.H[2] * s1));
        I0t = cur.I0;
        ret = qre;
        nt = qn;
    }
    FitOut out;
    out.I0 = cur.I0;
    out.re = re;
    out.n = n;
    out.chi2 = cur.chi2;
    bool refined = false;
    if (isfinite(cur.chi2) && re > re_min && re < re_max && n > n_min && n < n_max) {
        // Newton refinement on exact chi^2 (double-float sums): the error left
        // after a step is about the square of the step, so a step below 1e-4
        // (relative; about 1e-8 left) ends it, applied with chi^2 from the
        // quadratic model (exact to third order in the step).  The fp32
        // iteration above therefore stops at a 1e-4 step (tol_fit) and leaves
        // the last stretch to this quadratically converging pass.  Steps up to
        // 1e-2 are taken as they are; larger ones are capped at 20 % of each
        // parameter and taken only if the exact chi^2 does not rise, else
        // retried at a quarter of the length.  This also finishes fits that
        // the fp32 iteration left early in a flat valley, where chi^2 changes
        // below its fp32 resolution.
        // one call site (the pixel pass is large): each round evaluates the
        // next point, then accepts or rejects it against the best so far
        Precise P;
        P.ok = false;
        float te = re, tn = n, tI0 = cur.I0;   // the point to evaluate next
        float step_last = 0.f;                  // relative length of the step to it
        float shrink = 1.f;
        int passes = 0;
#pragma unroll 1
        for (;;) {
            const Precise E = fit_refine<IVAR, NW, SUP>(s, L, sq, w, npix, g, tI0, te, tn, lq, st, S);
            ++passes;
            // a step within 1e-2 is taken on the Newton model alone: its chi^2
            // decrease can be below the rounding of the fp32 model values
            const bool accept = passes == 1 || (E.ok && (step_last <= kFitRefineTrusted || E.chi2 <= P.chi2));
            if (accept) {
                P = E;
                re = te;
                n = tn;
                shrink = 1.f;
            } else {
                shrink *= 0.25f;
                if (shrink < 1e-3f) break;
            }
            if (!P.ok) break;
            const float rel = fmaxf(fabsf(P.d0) / re, fabsf(P.d1) / n);
            if (rel <= kFitRefineSkip) {
                out.re = re + P.d0;
                out.n = n + P.d1;
                out.I0 = P.I0 + P.c0 * P.d0 + P.c1 * P.d1;
                out.chi2 = P.chi2_step;
                refined = true;
                break;
            }
            if (passes >= kFitRefineMax) break;
            const float f = fminf(1.f, kFitRefineCap / rel) * shrink;
            te = re + f * P.d0;
            tn = n + f * P.d1;
            te = te < re_min ? re_min : (te > re_max ? re_max : te);
            tn = tn < n_min ? n_min : (tn > n_max ? n_max : tn);
            tI0 = P.I0 + P.c0 * (te - re) + P.c1 * (tn - n);
            step_last = f * rel;
        }
        if (!refined) {
            // no step small enough to end on: keep the best point evaluated
            out.re = re;
            out.n = n;
            if (isfinite(P.chi2)) {
                out.I0 = P.I0;
                out.chi2 = P.chi2;
            }
        }
        if (passes > 1) status |= FSE_ST_FIT_REFINE2;
    }
    if ((converged || refined) && isfinite(out.chi2)) status |= FSE_ST_FIT_CONVERGED;
    else if (finite0 && it > o.max_iter_fit) status |= FSE_ST_FIT_MAXITER;
    if (out.re <= re_min || out.re >= re_max || out.n <= n_min || out.n >= n_max)
        status |= FSE_ST_FIT_BOUND;
    if (!(out.I0 > 0.f)) status |= FSE_ST_NONPOS_FLUX;
    out.iters = evals;
    float b, db;
    bn_eval_f(out.n, &b, &db);
    const float q = (1.f - gabs) / (1.f + gabs);
    out.flux = 2.f * static_cast<float>(kPi) * out.n *
               expf(lgammaf(2.f * out.n) - 2.f * out.n * logf(b)) * out.I0 * out.re * out.re * q;
    return out;
}

// ------------------------------------------------------------------ kernel
// NW warps share each stamp (a stamp group); a CTA holds blockDim.x / (32 NW)
// groups, each with its own tile and, for NW > 1, named barrier 1 + group.
template <int STAGE, int DT, bool IVAR, int NW, bool SUP = false>
// Fit stages: 168 registers per thread let three CTAs of four warps share an
// SM (the launch shape of 48x48 and smaller tiles); more would leave two.
// Moment stages and the start-up: 96 registers (they spill nothing at 96) let
// five CTAs of four warps share an SM with their compact tile.  With eight
// warps per stamp (the 128x128 tiles) the tile already limits an SM to two
// CTAs of 256 threads, so 128 registers cost no occupancy and keep the group
// reductions of the refinement pass out of local memory.
__global__ void __maxnreg__(moment_stage(STAGE) ? (NW >= 8 ? 128 : 96) : 168) estimator_kernel(LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int grp = warp / NW;
    Grp<NW> g;
    g.lane = lane;
    g.wi = warp - grp * NW;
    g.t = g.wi * 32 + lane;
    g.bar = 1 + grp;
    const int max_pix = a.opts.max_pix;
    constexpr bool kBf16 = DT == FSE_BF16;
    constexpr bool kIv = IVAR && !moment_stage(STAGE);   // the moments do not use inverse variance
    const int slots = a.opts.ring_slots;
    const size_t wb = stage_warp_bytes(STAGE, max_pix, kBf16, IVAR, slots);
    unsigned char* wbase =
        smem + static_cast<size_t>(grp) * stage_group_bytes(STAGE, max_pix, kBf16, IVAR, NW, slots);
    float* pixbuf = reinterpret_cast<float*>(wbase);
    float* aux = reinterpret_cast<float*>(wbase + pix_bytes(max_pix));
    float* ivbuf = kIv ? reinterpret_cast<float*>(wbase + pix_bytes(max_pix) +
                                                  stage_aux_bytes(STAGE, max_pix, kBf16, slots))
                       : nullptr;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wbase + wb - 16);
    g.red = reinterpret_cast<float*>(wbase + wb);   // used when NW > 1
    unsigned* slot = reinterpret_cast<unsigned*>(wbase + wb + NW * 128);
    if (g.t == 0) mbar_init(bar);
    g.sync();
    if (g.t == 0) fence_proxy_async();
    g.sync();
    uint32_t phase = 0;
    const DevOpts& o = a.opts;
    // this launch's stamps: all of them, or one size class through perm
    const unsigned long long count = a.range ? a.range[1] : static_cast<unsigned long long>(a.count);
    const unsigned base = a.range ? a.range[0] : 0u;

    for (int round = 0;; ++round) {
        unsigned sidx = 0;
        if (a.static_assign) {
            // one stamp per group, no work counter (used by the per-stamp launches)
            if (round > 0) break;
            sidx = blockIdx.x * (blockDim.x / Grp<NW>::NT) + grp;
        } else if (NW == 1) {
            if (lane == 0) sidx = atomicAdd(a.queue, 1u);
            sidx = __shfl_sync(kFull, sidx, 0);
        } else {
            g.sync();   // the whole group has read the previous stamp's word
            if (g.t == 0) *slot = atomicAdd(a.queue, 1u);
            g.sync();
            sidx = *slot;
        }
        if (sidx >= count) break;
        const int64_t si = a.perm ? static_cast<int64_t>(a.perm[base + sidx]) : static_cast<int64_t>(sidx);
        const fse_stamp ix = a.idx[si];
        const int h = ix.h, w = ix.w;
        const long long npl = static_cast<long long>(h) * w;
        fse_result res;
        if (STAGE == kStageStartup) {
            res = fse_result{};
        } else {
            res = a.out[si];
        }
        uint32_t status = STAGE == kStageStartup
                              ? 0u
                              : (res.status & (FSE_ST_SIGW_CLAMPED | FSE_ST_INIT_FALLBACK |
                                               (STAGE == kStageFit ? (FSE_ST_MOM_CONVERGED |
                                                                      FSE_ST_MOM_MAXITER)
                                                                   : 0u)));
        bool skip = false;
        if (STAGE == kStageCentroid || STAGE == kStageMoments) {
            // the record of the start-up launch: a stamp it refused keeps that
            // record as it is
            status = res.status;
            if (status & (FSE_ST_BAD_SIZE | FSE_ST_NONFINITE | FSE_ST_TIMEOUT)) {
                g.sync();   // every thread has read the record
                continue;
            }
        }
        // the centre as the moment stage holds it (integer + fraction, finer
        // than the float x0 of the record), handed from the first launch of the
        // chain to the second in the record's fit fields
        int chain_xi = 0, chain_yi = 0;
        float chain_xf = 0.f, chain_yf = 0.f;
        if (STAGE == kStageFit && a.chain_fit) {
            // the second launch of the chain: the record is this launch's own
            // first half; its bits stay, and only converged moments are fitted
            status = res.status & ~(FSE_ST_FIT_CONVERGED | FSE_ST_FIT_MAXITER | FSE_ST_FIT_BOUND |
                                    FSE_ST_FIT_SINGULAR | FSE_ST_NONPOS_FLUX | FSE_ST_FIT_REFINE2);
            if (!(status & FSE_ST_MOM_CONVERGED) ||
                (status & (FSE_ST_BAD_SIZE | FSE_ST_NONFINITE | FSE_ST_TIMEOUT))) {
                g.sync();   // every thread has read the record before it is rewritten
                continue;
            }
            chain_xi = __float_as_int(res.I0);
            chain_yi = __float_as_int(res.re);
            chain_xf = res.n;
            chain_yf = res.flux;
            res.I0 = res.re = res.n = res.flux = 0.f;
        }
        res.npix = static_cast<int32_t>(npl > 0x7fffffff ? 0x7fffffff : npl);
        if (h < 1 || w < 1 || h > FSE_MAX_SIDE || w > FSE_MAX_SIDE || npl > max_pix) {
            status |= FSE_ST_BAD_SIZE;
            skip = true;
        }
        float* s = pixbuf;
        if (!skip) {
            const char* gsrc = static_cast<const char*>(a.pix) + ix.offset * (DT == FSE_BF16 ? 2 : 4);
            const float scale = (DT == FSE_BF16 && a.scale) ? a.scale[si] : 1.f;
            const bool ok = stage_stamp<DT>(pixbuf, &s, aux, gsrc, static_cast<int>(npl), scale, bar,
                                            &phase, g);
            if (kIv && ok) {
                const float* gv = a.inv_var + ix.offset;
                for (int p = g.t; p < npl; p += Grp<NW>::NT) ivbuf[p] = sqrtf(fmaxf(__ldg(gv + p), 0.f));
                g.sync();
            }
            if (!ok) {
                // the copy did not complete within the bound: report and stop this
                // group (the verdict is the same in all its threads)
                if (g.t == 0) {
                    atomicOr(a.err, 1u);
                    res.status = status | FSE_ST_TIMEOUT;
                    a.out[si] = res;
                }
                return;
            }
        }
        const int npix = static_cast<int>(npl);
        MomState st;
        if (STAGE == kStageStartup) {
            // the start-up of Sec. 4.1, recorded for the moment launch: the
            // brightest pixel (as x0, y0), r50 and the weight size it gives
            if (!skip) {
                const InitOut in = stamp_init(s, h, w, npix, g, reinterpret_cast<unsigned*>(aux), slots);
                if (!in.finite) {
                    status |= FSE_ST_NONFINITE;
                } else if (in.overflow) {
                    status |= FSE_ST_BAD_SIZE;
                } else {
                    if (in.fallback) status |= FSE_ST_INIT_FALLBACK;
                    float sw = in.r50 / static_cast<float>(kSqrt2Ln2);
                    const float smax = 0.5f * static_cast<float>(h < w ? h : w);
                    if (sw < 0.5f) { sw = 0.5f; status |= FSE_ST_SIGW_CLAMPED; }
                    if (sw > smax) { sw = smax; status |= FSE_ST_SIGW_CLAMPED; }
                    res.x0 = static_cast<float>(in.peak % w);
                    res.y0 = static_cast<float>(in.peak / w);
                    res.r50 = in.r50;
                    res.sigma_w = sw;
                }
            }
            res.status = status;
            if (g.t == 0) a.out[si] = res;
            g.sync();
            continue;
        }
        if (!skip && (STAGE == kStageCentroid || STAGE == kStageMoments)) {
            // start at the brightest pixel with the start-up's weight size
            st.xi = static_cast<int>(res.x0);
            st.yi = static_cast<int>(res.y0);
            st.xf = st.yf = 0.f;
            st.g1 = st.g2 = 0.f;
            st.sw = res.sigma_w;
        } else if (!skip) {
            // centre (and for the fit, ellipticity) from the previous stage
            bool fin = true;
            for (int p = g.t; p < npix; p += Grp<NW>::NT) fin = fin && isfinite(s[p]);
            if (!g.all(fin)) {
                status |= FSE_ST_NONFINITE;
                skip = true;
            }
            const float rx = rintf(res.x0), ry = rintf(res.y0);
            st.xi = static_cast<int>(rx);
            st.yi = static_cast<int>(ry);
            st.xf = res.x0 - rx;
            st.yf = res.y0 - ry;
            if (STAGE == kStageFit && a.chain_fit) {
                st.xi = chain_xi;
                st.yi = chain_yi;
                st.xf = chain_xf;
                st.yf = chain_yf;
            }
            st.g1 = STAGE == kStageFit ? res.e1 : 0.f;
            st.g2 = STAGE == kStageFit ? res.e2 : 0.f;
            st.sw = res.sigma_w;
            if (!(st.sw > 0.f) || !isfinite(res.x0) || !isfinite(res.y0)) {
                status |= FSE_ST_MOM_FAILED;
                skip = true;
            }
        }
        if (!skip && STAGE != kStageFit) {
            const bool ellip = STAGE != kStageCentroid;
            res.it_mom = moment_iterate(s, h, w, npix, g, o, ellip, st, status);
            res.x0 = static_cast<float>(st.xi) + st.xf;
            res.y0 = static_cast<float>(st.yi) + st.yf;
            res.sigma_w = st.sw;
            if (ellip) {
                res.e1 = st.g1;
                res.e2 = st.g2;
            }
            if (!(status & FSE_ST_MOM_CONVERGED)) skip = true;
            if (STAGE == kStageMoments && !skip) {
                // for the chain's fit launch, which clears these fields first
                res.I0 = __int_as_float(st.xi);
                res.re = __int_as_float(st.yi);
                res.n = st.xf;
                res.flux = st.yf;
            }
        }
        if (!skip && (STAGE == kStageFit || STAGE == kStageAll)) {
            const FitOut f = sersic_fit<IVAR, NW, SUP>(s, aux, ivbuf, h, w, npix, g, o, st, status);
            res.I0 = static_cast<float>(f.I0);
            res.re = static_cast<float>(f.re);
            res.n = static_cast<float>(f.n);
            res.flux = static_cast<float>(f.flux);
            res.chi2 = f.chi2;
            res.it_fit = f.iters;
        }
        res.status = status;
        if (g.t == 0) a.out[si] = res;
        g.sync();
    }
}

template <int STAGE, int DT, bool IVAR, int NW, bool SUP = false>
cudaError_t launch_t(const LaunchArgs& a_in, cudaStream_t stream) {
    LaunchArgs a = a_in;
    a.opts.ring_slots = ring_slots(a.opts.max_pix);
    const int groups = a.warps_per_cta / NW;
    if (groups < 1 || groups * NW != a.warps_per_cta || groups > 15) return cudaErrorInvalidValue;
    const size_t smem =
        stage_group_bytes(STAGE, a.opts.max_pix, DT == FSE_BF16, IVAR, NW, a.opts.ring_slots) * groups;
    auto kern = estimator_kernel<STAGE, DT, IVAR, NW, SUP>;
    // the shared-memory opt-in is raised once per instantiation and size (per
    // device and context: a device reset clears it)
    static size_t opted[64] = {0};
    static unsigned long long opted_ctx[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev >= 64) return e != cudaSuccess ? e : cudaErrorInvalidDevice;
    const unsigned long long cid = current_context_id();
    if (cid != opted_ctx[dev]) {
        opted[dev] = 0;
        opted_ctx[dev] = cid;
    }
    if (smem > opted[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        opted[dev] = smem;
    }
    long long grid = a.num_ctas;
    if (grid <= 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * a.warps_per_cta, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = static_cast<long long>(per_sm) * sms;
    }
    const long long need = (a.count + groups - 1) / groups;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), 32 * a.warps_per_cta, smem, stream>>>(a);
    return cudaGetLastError();
}

// Warps per stamp: several only for the whole chain (the large-stamp launches
// of the ragged path); the single stages keep one warp per stamp.
template <int STAGE, int DT, bool IVAR>
cudaError_t launch_nw(const LaunchArgs& a, cudaStream_t stream) {
    const int nw = a.warps_per_stamp > 1 ? a.warps_per_stamp : 1;
    if constexpr (STAGE == kStageFit) {
        // the pixel-integrated model: one warp per stamp
        if (a.opts.supersample > 1) {
            if (nw != 1) return cudaErrorInvalidValue;
            return launch_t<STAGE, DT, IVAR, 1, true>(a, stream);
        }
    }
    // several warps per stamp: the three launches of the whole chain
    if constexpr (STAGE == kStageMoments || STAGE == kStageFit || STAGE == kStageStartup) {
        switch (nw) {
            case 1: return launch_t<STAGE, DT, IVAR, 1>(a, stream);
            case 2: return launch_t<STAGE, DT, IVAR, 2>(a, stream);
            case 4: return launch_t<STAGE, DT, IVAR, 4>(a, stream);
            case 8: return launch_t<STAGE, DT, IVAR, 8>(a, stream);
            default: return cudaErrorInvalidValue;
        }
    } else {
        if (nw != 1) return cudaErrorInvalidValue;
        return launch_t<STAGE, DT, IVAR, 1>(a, stream);
    }
}

template <int STAGE>
cudaError_t launch_stage(const LaunchArgs& a, cudaStream_t stream) {
    if constexpr (moment_stage(STAGE)) {
        // the moment stages and the start-up do not read the inverse variance
        if (a.dtype == FSE_BF16) return launch_nw<STAGE, FSE_BF16, false>(a, stream);
        return launch_nw<STAGE, FSE_F32, false>(a, stream);
    } else {
        const bool iv = a.inv_var != nullptr;
        if (a.dtype == FSE_BF16)
            return iv ? launch_nw<STAGE, FSE_BF16, true>(a, stream) : launch_nw<STAGE, FSE_BF16, false>(a, stream);
        return iv ? launch_nw<STAGE, FSE_F32, true>(a, stream) : launch_nw<STAGE, FSE_F32, false>(a, stream);
    }
}

}  // namespace

// ------------------------------------------------------------------ host wrappers
unsigned long long current_context_id() {
    // the driver's cuCtxGetCurrent and cuCtxGetId, looked up through the
    // runtime (no link dependency on the driver library)
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

size_t smem_per_group(int max_pix, bool ivar, int warps_per_stamp) {
    return group_bytes(max_pix, ivar, warps_per_stamp);
}

void choose_launch(int max_pix, int* warps_per_cta, int* warps_per_stamp) {
    // one warp per stamp up to 48x48 tiles; larger tiles leave room for few
    // stamps per SM, so several warps share each of them
    const int nw = max_pix <= 48 * 48 ? 1 : max_pix <= 64 * 64 ? 2 : max_pix <= 96 * 96 ? 4 : 8;
    const size_t spg = group_bytes(max_pix, false, nw);
    const size_t budget = 227 * 1024;
    int groups = nw == 1 ? 4 : 1;
    while (groups > 1 && spg * groups > budget) groups >>= 1;
    *warps_per_cta = groups * nw;
    *warps_per_stamp = nw;
}

const float2* bn_table_f32() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bnf) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<const float2*>(p);
}

cudaError_t build_bn_table(cudaStream_t stream) {
    build_bn_kernel<<<(kBnNodes + 127) / 128, 128, 0, stream>>>();
    return cudaGetLastError();
}

cudaError_t eval_bn(const double* n, double* b, double* db, int64_t count, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    eval_bn_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, stream>>>(n, b, db, count);
    return cudaGetLastError();
}

// The start-up launch before a moment launch on the same stream; the work
// counter is cleared between the two.
static cudaError_t launch_startup(const LaunchArgs& a, cudaStream_t stream) {
    LaunchArgs u = a;
    u.stage = kStageStartup;
    cudaError_t e = launch_stage<kStageStartup>(u, stream);
    if (e != cudaSuccess || a.static_assign) return e;
    return cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), stream);
}

cudaError_t launch_estimator(const LaunchArgs& a, cudaStream_t stream) {
    switch (a.stage) {
        case kStageCentroid: {
            cudaError_t e = launch_startup(a, stream);
            if (e != cudaSuccess) return e;
            return launch_stage<kStageCentroid>(a, stream);
        }
        case kStageEllipticity: return launch_stage<kStageEllipticity>(a, stream);
        case kStageFit: return launch_stage<kStageFit>(a, stream);
        default: {
            // The whole chain as three persistent launches on the same stream:
            // the start-up, the moment iteration, then the fit of the stamps
            // whose moments converged.  Each kernel holds only its own phase's
            // code (instruction fetch stalls grow with a kernel's code), its
            // registers and its tile; the pixels are read from HBM once per
            // launch.
            cudaError_t e = launch_startup(a, stream);
            if (e != cudaSuccess) return e;
            LaunchArgs m = a;
            m.stage = kStageMoments;
            e = launch_stage<kStageMoments>(m, stream);
            if (e != cudaSuccess) return e;
            if (!a.static_assign) {
                e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), stream);
                if (e != cudaSuccess) return e;
            }
            LaunchArgs f = a;
            f.stage = kStageFit;
            f.chain_fit = 1;
            return launch_stage<kStageFit>(f, stream);
        }
    }
}

}  // namespace fse
