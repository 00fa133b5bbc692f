// fse_api.cu -- the C ABI of libfse (declared in include/fse.h): context,
// argument checks, launch selection, the host-buffer pipeline and the
// per-stamp launch form.  No computation of the method happens here; every
// step of the estimator runs in the kernels of fse_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fse.h"
#include "fse_internal.h"

// Chunks of the host-buffer pipeline (fse_fit_batch_host), in units of 1/64
// of the batch.  The kernels start after the copy of the small first chunk;
// the chunks then grow while the copy runs ahead of the kernels, level off,
// and shrink again so that little compute is left once the last copy is done.
// The host link's rate differs between machines (211 GB/s measured on one
// GB300 host; another behaved as about 120 GB/s, against about 100 GB/s of
// pixels consumed by the kernels on 48x48 stamps), and by a model of the
// pipeline this schedule stays within 10% of the best over that range; few chunks, because every chunk adds two launch tails
// (on 100,000 stamps of 48x48, twelve chunks cost 11.0 ms against 9.5 ms for
// one launch pair).
constexpr int kHostChunks = 9;
constexpr int kChunkUnits[kHostChunks] = {2, 4, 6, 8, 10, 10, 10, 8, 6};
constexpr int chunk_units_total() {
    int t = 0;
    for (int u : kChunkUnits) t += u;
    return t;
}
static_assert(chunk_units_total() == 64, "the chunks must cover the batch in 64ths");

struct fse_ctx {
    int device = 0;
    char err[512] = {0};
    unsigned int* d_queue = nullptr;   // kQueues work counters
    unsigned int* d_err = nullptr;     // sticky error word written by the kernels
    unsigned next_queue = 0;
    cudaStream_t aux_stream = nullptr; // second compute stream of the host-buffer pipeline
    cudaStream_t copy_stream = nullptr; // host-to-device copies of the host-buffer pipeline
    cudaEvent_t chunk_ev[kHostChunks + 2] = {}; // chunk copies done; start; end
    // grow-only device staging of fse_fit_batch_host
    void* d_pix = nullptr;
    size_t pix_cap = 0;
    fse_stamp* d_idx = nullptr;
    size_t idx_cap = 0;
    fse_result* d_out = nullptr;
    size_t out_cap = 0;
    float* d_scale = nullptr;
    size_t scale_cap = 0;
    float* d_ivar = nullptr;
    size_t ivar_cap = 0;
    // ragged path: stamps grouped by size class, and the class bookkeeping
    // (counts[K] | range[2K] | cursor[K] | work counters[K])
    int32_t* d_perm = nullptr;
    size_t perm_cap = 0;
    unsigned int* d_cls = nullptr;
    // grow-only per-stamp coefficients of fse_moment_vjp, and growth-curve
    // records of fse_moment_vjp / _jvp
    fse::VjpCoef* d_vjp = nullptr;
    size_t vjp_cap = 0;
    fse::R50Grad* d_r50 = nullptr;
    size_t r50_cap = 0;
    // warps per CTA chosen by fse_autotune, by dtype, inverse variance and size
    // class (0 = library default)
    int tuned[2][2][fse::kClasses] = {};
    int tuned_nw[2][2][fse::kClasses] = {};   // warps per stamp of the tuned shape
    unsigned tune_version = 0;
    // the CUDA graph of the last ragged call made with FSE_FLAG_GRAPH
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned char gkey[256] = {0};
};

namespace {

constexpr int kQueues = 64;
std::mutex g_table_mutex;
// the context in which each device's b(n) table was built (0: not built); a
// device reset makes a new primary context, whose table is built again
unsigned long long g_table_ctx[256];
bool g_table_built[256];

// Build the b(n) table of the current device unless it exists in the current
// context.  Synchronises the device when it builds.  Call under g_table_mutex.
cudaError_t ensure_bn_table(int device) {
    if (g_table_built[device] && g_table_ctx[device] == fse::current_context_id()) return cudaSuccess;
    cudaError_t e = fse::build_bn_table(nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    g_table_built[device] = true;
    g_table_ctx[device] = fse::current_context_id();   // the launch made the context current
    return cudaSuccess;
}

int set_error(fse_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(fse_ctx* ctx, cudaError_t e, const char* what) {
    return set_error(ctx, FSE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes ctx->device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_opts(fse_ctx* ctx, const fse_opts* o) {
    if (o->size != sizeof(fse_opts)) return set_error(ctx, FSE_EINVAL, "opts.size must be sizeof(fse_opts)");
    if (!(o->tol_pos > 0 && o->tol_g > 0 && o->tol_sig > 0 && o->tol_fit > 0))
        return set_error(ctx, FSE_EINVAL, "tolerances must be positive");
    if (o->max_iter_mom < 1 || o->max_iter_mom > 100000 || o->max_iter_fit < 1 || o->max_iter_fit > 100000)
        return set_error(ctx, FSE_EINVAL, "max_iter must be in [1, 100000]");
    if (!(o->k_gain >= 0 && o->k_gain <= 4)) return set_error(ctx, FSE_EINVAL, "k_gain must be in [0, 4]");
    if (o->sigw_mode != 0 && o->sigw_mode != 1) return set_error(ctx, FSE_EINVAL, "sigw_mode must be 0 or 1");
    if (o->max_pix < 0 || o->max_pix > FSE_MAX_PIX)
        return set_error(ctx, FSE_EINVAL, "max_pix must be in [0, %d]", FSE_MAX_PIX);
    const double tab_lo = fse::kBnLo + 2 * fse::kBnStep;
    const double tab_hi = fse::kBnLo + (fse::kBnNodes - 3) * fse::kBnStep;
    if (!(o->n_min >= tab_lo && o->n_max <= tab_hi && o->n_min < o->n_max))
        return set_error(ctx, FSE_EINVAL, "n bounds must satisfy %.4f <= n_min < n_max <= %.4f", tab_lo, tab_hi);
    if (!(o->re_min > 0 && o->re_max_frac > 0)) return set_error(ctx, FSE_EINVAL, "r_e bounds must be positive");
    if (!(o->lm_lambda0 > 0)) return set_error(ctx, FSE_EINVAL, "lm_lambda0 must be positive");
    const int w = o->warps_per_cta, ws = o->warps_per_stamp;
    if (!(w == 0 || w == 1 || w == 2 || w == 4 || w == 8))
        return set_error(ctx, FSE_EINVAL, "warps_per_cta must be 0, 1, 2, 4 or 8");
    if (!(ws == 0 || ws == 1 || ws == 2 || ws == 4 || ws == 8))
        return set_error(ctx, FSE_EINVAL, "warps_per_stamp must be 0, 1, 2, 4 or 8");
    if (w > 0 && ws > 0 && w % ws != 0)
        return set_error(ctx, FSE_EINVAL, "warps_per_cta must be a multiple of warps_per_stamp");
    if (o->flags & ~static_cast<uint32_t>(FSE_FLAG_GRAPH))
        return set_error(ctx, FSE_EINVAL, "unknown bits in flags");
    if (o->supersample < 0 || o->supersample > 8) return set_error(ctx, FSE_EINVAL, "supersample must be in [0, 8]");
    if (o->supersample > 1 && ws > 1)
        return set_error(ctx, FSE_EINVAL, "supersample > 1 runs one warp per stamp (warps_per_stamp 0 or 1)");
    return FSE_OK;
}

fse::DevOpts dev_opts(const fse_opts& o) {
    fse::DevOpts d;
    d.tol_pos = static_cast<float>(o.tol_pos);
    d.tol_g = static_cast<float>(o.tol_g);
    d.tol_sig = static_cast<float>(o.tol_sig);
    d.tol_fit = static_cast<float>(o.tol_fit);
    d.max_iter_mom = o.max_iter_mom;
    d.max_iter_fit = o.max_iter_fit;
    d.k_gain = static_cast<float>(o.k_gain);
    d.sigw_mode = o.sigw_mode;
    d.max_pix = o.max_pix > 0 ? o.max_pix : FSE_MAX_PIX;
    d.n_min = static_cast<float>(o.n_min);
    d.n_max = static_cast<float>(o.n_max);
    d.re_min = static_cast<float>(o.re_min);
    d.re_max_frac = static_cast<float>(o.re_max_frac);
    d.lm_lambda0 = static_cast<float>(o.lm_lambda0);
    d.supersample = o.supersample > 1 ? o.supersample : 1;
    return d;
}

// Launch shape for a tile: the options' warps per CTA and per stamp where
// given, the library choice otherwise.  Only the whole chain puts several
// warps on a stamp; a warps_per_cta given alone means one warp per stamp.
void launch_shape(const fse_opts& o, int max_pix, int stage, int* wpc, int* nw) {
    int dw = 0, dn = 0;
    fse::choose_launch(max_pix, &dw, &dn);
    int n = o.warps_per_stamp > 0 ? o.warps_per_stamp : (o.warps_per_cta > 0 ? 1 : dn);
    if (stage != fse::kStageAll || o.supersample > 1) n = 1;
    int w = o.warps_per_cta > 0 ? o.warps_per_cta : (n == dn ? dw : n);
    if (n == 1 && o.warps_per_cta <= 0 && dn != 1) {
        // one warp per stamp on a large tile: as many as fit, up to four
        const size_t spw = fse::smem_per_group(max_pix, false, 1);
        w = 4;
        while (w > 1 && spw * w > 227 * 1024) w >>= 1;
    }
    *wpc = w;
    *nw = n;
}

// Common checks of the device entry points; fills `a` on success.
int prepare(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
            int64_t count, const float* inv_var, const fse_opts* opts, fse_result* out, int stage,
            fse::LaunchArgs* a) {
    if (!ctx) return FSE_EINVAL;
    if (count < 0 || count > 0x7fffffffLL) return set_error(ctx, FSE_EINVAL, "count out of range");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    fse_opts def;
    fse_opts_default(&def);
    const fse_opts& o = opts ? *opts : def;
    int rc = check_opts(ctx, &o);
    if (rc) return rc;
    if (count > 0) {
        if (!pix || !idx || !out) return set_error(ctx, FSE_EINVAL, "pix, idx and out must not be NULL");
        if (!is_device_ptr(pix) || !is_device_ptr(idx) || !is_device_ptr(out) ||
            (scale && !is_device_ptr(scale)) || (inv_var && !is_device_ptr(inv_var)))
            return set_error(ctx, FSE_EINVAL, "pix, scale, idx, inv_var and out must be device pointers");
    }
    memset(a, 0, sizeof *a);
    a->pix = pix;
    a->dtype = dtype;
    a->scale = scale;
    a->idx = idx;
    a->count = count;
    a->inv_var = inv_var;
    a->out = out;
    a->err = ctx->d_err;
    a->opts = dev_opts(o);
    a->stage = stage;
    if (stage != fse::kStageAll && o.warps_per_stamp > 1)
        return set_error(ctx, FSE_EINVAL, "warps_per_stamp > 1 applies to the whole chain only");
    launch_shape(o, a->opts.max_pix, stage, &a->warps_per_cta, &a->warps_per_stamp);
    if (a->warps_per_cta % a->warps_per_stamp != 0)
        return set_error(ctx, FSE_EINVAL, "warps_per_cta must be a multiple of warps_per_stamp");
    return FSE_OK;
}

int run(fse_ctx* ctx, fse::LaunchArgs& a, cudaStream_t stream) {
    if (a.count == 0) return FSE_OK;
    a.queue = ctx->d_queue + (ctx->next_queue++ % kQueues);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "work counter reset");
    e = fse::launch_estimator(a, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "estimator launch");
    return FSE_OK;
}

int stage_entry(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                int64_t count, const float* inv_var, const fse_opts* opts, fse_result* out,
                void* stream, int stage) {
    if (!ctx) return FSE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    fse::LaunchArgs a;
    int rc = prepare(ctx, pix, dtype, scale, idx, count, inv_var, opts, out, stage, &a);
    if (rc) return rc;
    return run(ctx, a, static_cast<cudaStream_t>(stream));
}

template <typename T>
int grow(fse_ctx* ctx, T** p, size_t* cap, size_t n) {
    if (n <= *cap) return FSE_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, FSE_ENOMEM, "device staging of %zu bytes: %s", n * sizeof(T),
                         cudaGetErrorString(e));
    }
    *cap = n;
    return FSE_OK;
}

// ---------------------------------------------------------------- ragged path
constexpr int kK = fse::kClasses;

int ragged_workspace(fse_ctx* ctx, int64_t count) {
    int rc = grow(ctx, &ctx->d_perm, &ctx->perm_cap, static_cast<size_t>(count));
    if (rc) return rc;
    if (!ctx->d_cls) {
        cudaError_t e = cudaMalloc(&ctx->d_cls, 5 * kK * sizeof(unsigned int));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ctx, FSE_ENOMEM, "ragged workspace: %s", cudaGetErrorString(e));
        }
    }
    return FSE_OK;
}

// Launch shape of size class k: the options' where given, else the
// autotuner's choice, else the library default for the class's tile.
void class_shape(const fse_ctx* ctx, const fse::LaunchArgs& a, const fse_opts& o, int k, int* wpc,
                 int* nw) {
    if (o.warps_per_cta > 0 || o.warps_per_stamp > 0 || o.supersample > 1) {
        launch_shape(o, fse::kClassPix[k], fse::kStageAll, wpc, nw);
        return;
    }
    const int dt = a.dtype == FSE_BF16, iv = a.inv_var != nullptr;
    if (ctx->tuned[dt][iv][k] > 0) {
        *wpc = ctx->tuned[dt][iv][k];
        *nw = ctx->tuned_nw[dt][iv][k];
        return;
    }
    launch_shape(o, fse::kClassPix[k], fse::kStageAll, wpc, nw);
}

// Classification, then the chain's launch pair per size class (largest first),
// each with a shared-memory tile for its class.  Everything is stream-ordered
// on `s` with no host synchronisation, so the sequence can be captured.
int enqueue_ragged(fse_ctx* ctx, const fse::LaunchArgs& a, const fse_opts& o, cudaStream_t s) {
    unsigned int* counts = ctx->d_cls;
    unsigned int* range = counts + kK;
    unsigned int* cursor = range + 2 * kK;
    unsigned int* queues = cursor + kK;
    cudaError_t e = cudaMemsetAsync(counts, 0, kK * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(queues, 0, kK * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = fse::classify_stamps(a.idx, a.count, counts, range, cursor, ctx->d_perm, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "size classification");
    for (int k = kK - 1; k >= 0; --k) {
        fse::LaunchArgs b = a;
        b.opts.max_pix = fse::kClassPix[k];
        b.perm = ctx->d_perm;
        b.range = range + 2 * k;
        b.queue = queues + k;
        class_shape(ctx, a, o, k, &b.warps_per_cta, &b.warps_per_stamp);
        e = fse::launch_estimator(b, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "size-class launch");
    }
    return FSE_OK;
}

// Identity of a ragged call for the graph cache.
struct RaggedKey {
    const void* pix;
    const float* scale;
    const fse_stamp* idx;
    const float* inv_var;
    fse_result* out;
    const int32_t* perm;
    int64_t count;
    int dtype;
    unsigned tune_version;
    fse_opts opts;
};
static_assert(sizeof(RaggedKey) <= 256, "graph key");

void make_key(const fse_ctx* ctx, const fse::LaunchArgs& a, const fse_opts& o, RaggedKey* k) {
    memset(k, 0, sizeof *k);
    k->pix = a.pix;
    k->scale = a.scale;
    k->idx = a.idx;
    k->inv_var = a.inv_var;
    k->out = a.out;
    k->perm = ctx->d_perm;
    k->count = a.count;
    k->dtype = a.dtype;
    k->tune_version = ctx->tune_version;
    k->opts = o;
}

// Allocation-free form of fse_fit_batch (fse_fit_batch_static).  Some callers
// cannot allocate device memory at the point of the call: a service that must
// keep its footprint fixed after start-up, code running under a caching
// allocator that owns all of the device memory, or a caller that holds no
// fse_ctx.  The estimator's only per-call scratch is the work counter of the
// persistent launch and the error word of its bounded waits; for those callers
// both live in this file-scope array instead of in a context's device memory.
constexpr int kStaticWords = 2;                      // [0] work counter, [1] error word
constexpr int64_t kStaticMaxCount = 0x7fffffffLL;    // the 32-bit counter indexes at most this
static __device__ __align__(256) unsigned int g_static_scratch[kStaticWords];
unsigned int* g_static_addr[256];                    // its address on each device
unsigned long long g_static_ctx[256];                 // in the context it was looked up in

}  // namespace

extern "C" {

void fse_opts_default(fse_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->size = sizeof(fse_opts);
    o->tol_pos = 1e-6;
    o->tol_g = 1e-6;
    o->tol_sig = 1e-6;
    o->tol_fit = 1e-4;
    o->max_iter_mom = 60;
    o->max_iter_fit = 60;
    o->k_gain = 0.0;
    o->sigw_mode = 1;
    o->max_pix = 0;
    o->n_min = 0.2;
    o->n_max = 10.0;
    o->re_min = 0.2;
    o->re_max_frac = 2.0;
    o->lm_lambda0 = 1e-3;
    o->flags = 0;
    o->warps_per_cta = 0;
    o->warps_per_stamp = 0;
    o->supersample = 1;
}

int fse_create(fse_ctx** out, int device) {
    if (!out) return FSE_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev || device >= 256) {
        cudaGetLastError();
        return FSE_EINVAL;
    }
    fse_ctx* ctx = new fse_ctx();
    ctx->device = device;
    DeviceGuard g(device);
    if (!g.ok) { delete ctx; return FSE_ECUDA; }
    if (cudaMalloc(&ctx->d_queue, kQueues * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_err, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        fse_destroy(ctx);
        return FSE_ENOMEM;
    }
    if (cudaMemset(ctx->d_err, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        fse_destroy(ctx);
        return FSE_ECUDA;
    }
    for (cudaEvent_t& ev : ctx->chunk_ev) {
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            ev = nullptr;
            cudaGetLastError();
            fse_destroy(ctx);
            return FSE_ECUDA;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_table_mutex);
        if (ensure_bn_table(device) != cudaSuccess) {
            cudaGetLastError();
            fse_destroy(ctx);
            return FSE_ECUDA;
        }
    }
    *out = ctx;
    return FSE_OK;
}

void fse_destroy(fse_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        cudaFree(ctx->d_queue);
        cudaFree(ctx->d_err);
        cudaFree(ctx->d_pix);
        cudaFree(ctx->d_idx);
        cudaFree(ctx->d_out);
        cudaFree(ctx->d_scale);
        cudaFree(ctx->d_ivar);
        cudaFree(ctx->d_perm);
        cudaFree(ctx->d_cls);
        cudaFree(ctx->d_vjp);
        cudaFree(ctx->d_r50);
        if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
        if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        for (cudaEvent_t ev : ctx->chunk_ev)
            if (ev) cudaEventDestroy(ev);
        cudaGetLastError();
    }
    delete ctx;
}

const char* fse_last_error(const fse_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int fse_centroid(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                 int64_t count, const float* inv_var, const fse_opts* opts, fse_result* out,
                 void* stream) {
    return stage_entry(ctx, pix, dtype, scale, idx, count, inv_var, opts, out, stream,
                       fse::kStageCentroid);
}

int fse_ellipticity(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                    const fse_stamp* idx, int64_t count, const float* inv_var, const fse_opts* opts,
                    fse_result* inout, void* stream) {
    return stage_entry(ctx, pix, dtype, scale, idx, count, inv_var, opts, inout, stream,
                       fse::kStageEllipticity);
}

int fse_sersic_fit(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                   const fse_stamp* idx, int64_t count, const float* inv_var, const fse_opts* opts,
                   fse_result* inout, void* stream) {
    return stage_entry(ctx, pix, dtype, scale, idx, count, inv_var, opts, inout, stream,
                       fse::kStageFit);
}

int fse_fit_batch(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                  int64_t count, const float* inv_var, const fse_opts* opts, fse_result* out,
                  void* stream) {
    return stage_entry(ctx, pix, dtype, scale, idx, count, inv_var, opts, out, stream,
                       fse::kStageAll);
}

int fse_fit_batch_plain(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                        const fse_stamp* idx, int64_t count, const float* inv_var,
                        const fse_opts* opts, fse_result* out, void* stream) {
    if (!ctx) return FSE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    fse::LaunchArgs a;
    int rc = prepare(ctx, pix, dtype, scale, idx, count, inv_var, opts, out, fse::kStageAll, &a);
    if (rc) return rc;
    a.warps_per_cta = 1;
    a.warps_per_stamp = 1;
    a.num_ctas = 1;
    a.static_assign = 1;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int64_t i = 0; i < count; ++i) {
        fse::LaunchArgs b = a;
        b.idx = idx + i;
        b.out = out + i;
        b.count = 1;
        b.scale = scale ? scale + i : nullptr;
        cudaError_t e = fse::launch_estimator(b, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "per-stamp launch");
    }
    return FSE_OK;
}

int fse_fit_batch_host(fse_ctx* ctx, const void* pix, int64_t npix_total, int dtype,
                       const float* scale, const fse_stamp* idx, int64_t count,
                       const float* inv_var, const fse_opts* opts, fse_result* out, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count == 0) return FSE_OK;
    if (!pix || !idx || !out || count < 0 || count > 0x7fffffffLL || npix_total < 0)
        return set_error(ctx, FSE_EINVAL, "bad host arguments");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    fse_opts o;
    if (opts) o = *opts; else fse_opts_default(&o);
    int rc = check_opts(ctx, &o);
    if (rc) return rc;
    const size_t esz = dtype == FSE_BF16 ? 2 : 4;
    // chunk boundaries (stamps): one chunk below 8192 stamps, else the
    // kChunkUnits schedule
    int nchunk = 1;
    int64_t lo[kHostChunks + 1] = {0, count};
    if (count >= 8192) {
        nchunk = kHostChunks;
        int units = 0;
        for (int c = 0; c < kHostChunks; ++c) {
            lo[c] = count * units / 64;
            units += kChunkUnits[c];
        }
        lo[kHostChunks] = count;
    }
    if ((rc = grow(ctx, reinterpret_cast<char**>(&ctx->d_pix), &ctx->pix_cap, npix_total * esz)) ||
        (rc = grow(ctx, &ctx->d_idx, &ctx->idx_cap, count)) ||
        (rc = grow(ctx, &ctx->d_out, &ctx->out_cap, count)) ||
        (scale && (rc = grow(ctx, &ctx->d_scale, &ctx->scale_cap, count))) ||
        (inv_var && (rc = grow(ctx, &ctx->d_ivar, &ctx->ivar_cap, npix_total))))
        return rc;
    // Three streams: the copy stream moves every chunk's inputs to the device
    // back to back and records chunk_ev[c] after chunk c; chunk c's kernels and
    // its result copy run on compute stream c % 2 once chunk_ev[c] is done, so
    // one chunk's launch tail overlaps the next chunk's kernels.
    const cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    const cudaStream_t streams[2] = {s0, ctx->aux_stream};
    const cudaStream_t cs = ctx->copy_stream;
    cudaEvent_t ev_start = ctx->chunk_ev[kHostChunks], ev_end = ctx->chunk_ev[kHostChunks + 1];
    cudaError_t e = cudaEventRecord(ev_start, s0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux_stream, ev_start, 0);
    // First, chunk by chunk: every stamp inside the pixel buffer, the largest
    // stamp, the chunk's pixel span [p_lo, p_hi), then the chunk's copies, so
    // that the first chunks move while the later ones are checked.  From
    // pageable memory a copy returns only when done.
    int64_t maxp = 1;
    for (int c = 0; c < nchunk && e == cudaSuccess; ++c) {
        int64_t p_lo = INT64_MAX, p_hi = 0;
        for (int64_t st = lo[c]; st < lo[c + 1]; ++st) {
            const int64_t a = static_cast<int64_t>(idx[st].h) * idx[st].w;
            if (idx[st].h < 1 || idx[st].w < 1 || a > FSE_MAX_PIX) continue;
            if (idx[st].offset < 0 || idx[st].offset + a > npix_total) {
                cudaStreamSynchronize(cs);   // the copies already issued read the caller's buffers
                return set_error(ctx, FSE_EINVAL, "stamp %lld lies outside the pixel buffer", (long long)st);
            }
            maxp = std::max(maxp, a);
            p_lo = std::min(p_lo, idx[st].offset);
            p_hi = std::max(p_hi, idx[st].offset + a);
        }
        const int64_t s_lo = lo[c], n_c = lo[c + 1] - lo[c];
        if (n_c > 0) {
            e = cudaMemcpyAsync(ctx->d_idx + s_lo, idx + s_lo, n_c * sizeof(fse_stamp),
                                cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess && p_hi > p_lo)
                e = cudaMemcpyAsync(static_cast<char*>(ctx->d_pix) + p_lo * esz,
                                    static_cast<const char*>(pix) + p_lo * esz,
                                    (p_hi - p_lo) * esz, cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess && scale)
                e = cudaMemcpyAsync(ctx->d_scale + s_lo, scale + s_lo, n_c * sizeof(float),
                                    cudaMemcpyHostToDevice, cs);
            if (e == cudaSuccess && inv_var && p_hi > p_lo)
                e = cudaMemcpyAsync(ctx->d_ivar + p_lo, inv_var + p_lo,
                                    (p_hi - p_lo) * sizeof(float), cudaMemcpyHostToDevice, cs);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->chunk_ev[c], cs);
    }
    // Then each chunk's chain once its copy is done, all with the launch shape
    // of the batch's largest stamp (as fse_fit_batch, so the results are the same).
    if (o.max_pix == 0) o.max_pix = static_cast<int32_t>(maxp);
    for (int c = 0; c < nchunk && e == cudaSuccess; ++c) {
        const int64_t s_lo = lo[c], n_c = lo[c + 1] - lo[c];
        if (n_c == 0) continue;
        const cudaStream_t st = streams[c & 1];
        e = cudaStreamWaitEvent(st, ctx->chunk_ev[c], 0);
        if (e != cudaSuccess) break;
        fse::LaunchArgs a;
        memset(&a, 0, sizeof a);
        a.pix = ctx->d_pix;
        a.dtype = dtype;
        a.scale = scale ? ctx->d_scale + s_lo : nullptr;
        a.idx = ctx->d_idx + s_lo;
        a.count = n_c;
        a.inv_var = inv_var ? ctx->d_ivar : nullptr;
        a.out = ctx->d_out + s_lo;
        a.err = ctx->d_err;
        a.opts = dev_opts(o);
        a.stage = fse::kStageAll;
        launch_shape(o, a.opts.max_pix, fse::kStageAll, &a.warps_per_cta, &a.warps_per_stamp);
        rc = run(ctx, a, st);
        if (rc) {
            cudaStreamSynchronize(cs);
            cudaStreamSynchronize(ctx->aux_stream);
            cudaStreamSynchronize(s0);
            cudaGetLastError();
            return rc;
        }
        e = cudaMemcpyAsync(out + s_lo, ctx->d_out + s_lo, n_c * sizeof(fse_result),
                            cudaMemcpyDeviceToHost, st);
    }
    // the caller's stream waits for the other compute stream (whose work waited
    // on the copy stream's events), then the call waits for the caller's stream
    if (e == cudaSuccess) e = cudaEventRecord(ev_end, ctx->aux_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev_end, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamSynchronize(ctx->aux_stream);
        return cuda_fail(ctx, e, "host-buffer pipeline");
    }
    unsigned int flag = 0;
    e = cudaMemcpy(&flag, ctx->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word read");
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(unsigned int));
        return set_error(ctx, FSE_ETIMEOUT, "a bounded device wait expired");
    }
    return FSE_OK;
}

int fse_fit_batch_ragged(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                         const fse_stamp* idx, int64_t count, const float* inv_var,
                         const fse_opts* opts, fse_result* out, void* stream) {
    if (!ctx) return FSE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    fse_opts o;
    if (opts) o = *opts; else fse_opts_default(&o);
    fse::LaunchArgs a;
    int rc = prepare(ctx, pix, dtype, scale, idx, count, inv_var, &o, out, fse::kStageAll, &a);
    if (rc || count == 0) return rc;
    if ((rc = ragged_workspace(ctx, count))) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!(o.flags & FSE_FLAG_GRAPH)) return enqueue_ragged(ctx, a, o, s);
    RaggedKey key;
    make_key(ctx, a, o, &key);
    if (!ctx->gexec || memcmp(&key, ctx->gkey, sizeof key) != 0) {
        if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
        rc = enqueue_ragged(ctx, a, o, ctx->cap_stream);
        e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
        e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            ctx->gexec = nullptr;
            return cuda_fail(ctx, e, "graph instantiation");
        }
        memcpy(ctx->gkey, &key, sizeof key);
    }
    cudaError_t e = cudaGraphLaunch(ctx->gexec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    return FSE_OK;
}

int fse_autotune(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                 const fse_stamp* idx, int64_t count, const float* inv_var, const fse_opts* opts,
                 fse_result* out, void* stream) {
    if (!ctx) return FSE_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    fse_opts o;
    if (opts) o = *opts; else fse_opts_default(&o);
    fse::LaunchArgs a;
    int rc = prepare(ctx, pix, dtype, scale, idx, count, inv_var, &o, out, fse::kStageAll, &a);
    if (rc || count == 0) return rc;
    if ((rc = ragged_workspace(ctx, count))) return rc;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int* counts = ctx->d_cls;
    unsigned int* range = counts + kK;
    unsigned int* cursor = range + 2 * kK;
    unsigned int* queues = cursor + kK;
    cudaError_t e = cudaMemsetAsync(counts, 0, kK * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = fse::classify_stamps(a.idx, a.count, counts, range, cursor, ctx->d_perm, s);
    unsigned int hc[kK] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "size classification");
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    const int dt = dtype == FSE_BF16, iv = inv_var != nullptr;
    for (int k = 0; k < kK && e == cudaSuccess; ++k) {
        if (hc[k] == 0) continue;
        float best = 1e30f;
        int best_w = 0, best_n = 1;
        // (warps per stamp, stamp groups per CTA) with at most 8 warps per CTA
        // and the groups' tiles within the shared memory of a CTA
        for (int cand = 0; cand < 10 && e == cudaSuccess; ++cand) {
            static const int kNw[10] = {1, 1, 1, 1, 2, 2, 2, 4, 4, 8};
            static const int kGr[10] = {1, 2, 4, 8, 1, 2, 4, 1, 2, 1};
            const int nw = kNw[cand], groups = kGr[cand];
            if (nw > 1 && a.opts.supersample > 1) continue;
            if (fse::smem_per_group(fse::kClassPix[k], iv != 0, nw) * groups > 227 * 1024) continue;
            const int wpc = nw * groups;
            float t_min = 1e30f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                fse::LaunchArgs b = a;
                b.opts.max_pix = fse::kClassPix[k];
                b.perm = ctx->d_perm;
                b.range = range + 2 * k;
                b.queue = queues + k;
                b.warps_per_cta = wpc;
                b.warps_per_stamp = nw;
                e = cudaMemsetAsync(queues + k, 0, sizeof(unsigned int), s);
                if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
                if (e == cudaSuccess) e = fse::launch_estimator(b, s);
                if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
                if (e == cudaSuccess && ms < t_min) t_min = ms;
            }
            if (t_min < best) {
                best = t_min;
                best_w = wpc;
                best_n = nw;
            }
        }
        if (best_w > 0) {
            ctx->tuned[dt][iv][k] = best_w;
            ctx->tuned_nw[dt][iv][k] = best_n;
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune launch");
    ++ctx->tune_version;
    return FSE_OK;
}

int fse_tuned_warps(const fse_ctx* ctx, int dtype, int has_inv_var, int32_t* warps_per_cta,
                    int32_t* warps_per_stamp) {
    if (!ctx || !warps_per_cta || (dtype != FSE_F32 && dtype != FSE_BF16)) return FSE_EINVAL;
    fse_opts o;
    fse_opts_default(&o);
    for (int k = 0; k < kK; ++k) {
        const int dt = dtype == FSE_BF16, iv = has_inv_var != 0;
        int w = ctx->tuned[dt][iv][k], n = ctx->tuned_nw[dt][iv][k];
        if (w <= 0) launch_shape(o, fse::kClassPix[k], fse::kStageAll, &w, &n);
        warps_per_cta[k] = w;
        if (warps_per_stamp) warps_per_stamp[k] = n;
    }
    return FSE_OK;
}

// ---- the launch-shape cache of fse_autotune (fse_tuning_save / _load)
// One JSON object per line inside "entries", so that a saving process can keep
// the lines of other devices without a full JSON parser:
//   {"format": "libfse-launch-shapes/1", "entries": [
//   {"device": "<name>", "dtype": "f32", "inv_var": 0, "class_pix": [...7],
//    "warps_per_cta": [...7], "warps_per_stamp": [...7]},
//   ...
//   ]}
static const char kTuneFormat[] = "libfse-launch-shapes/1";

static bool device_name(int device, char* name, size_t len) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    snprintf(name, len, "%s", prop.name);
    for (char* c = name; *c; ++c)
        if (*c == '"' || *c == '\\' || static_cast<unsigned char>(*c) < 32) *c = '_';
    return true;
}

// The integers of the JSON array after `"key": [` in line, at most n of them.
static int json_ints(const char* line, const char* key, long* v, int n) {
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\": [", key);
    const char* p = strstr(line, pat);
    if (!p) return 0;
    p += strlen(pat);
    int k = 0;
    while (k < n) {
        char* end = nullptr;
        const long x = strtol(p, &end, 10);
        if (end == p) break;
        v[k++] = x;
        p = end;
        while (*p == ' ' || *p == ',') ++p;
        if (*p == ']') break;
    }
    return k;
}

static bool json_str(const char* line, const char* key, char* out, size_t len) {
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\": \"", key);
    const char* p = strstr(line, pat);
    if (!p) return false;
    p += strlen(pat);
    const char* q = strchr(p, '"');
    if (!q || static_cast<size_t>(q - p) >= len) return false;
    memcpy(out, p, q - p);
    out[q - p] = 0;
    return true;
}

int fse_tuning_save(const fse_ctx* ctx, const char* path) {
    if (!ctx || !path) return FSE_EINVAL;
    fse_ctx* c = const_cast<fse_ctx*>(ctx);
    char name[256];
    if (!device_name(ctx->device, name, sizeof name)) return set_error(c, FSE_ECUDA, "device properties");
    // the entries of other devices already in the file are kept
    std::vector<std::string> keep;
    if (FILE* f = fopen(path, "r")) {
        char line[4096];
        while (fgets(line, sizeof line, f)) {
            char dev[256];
            if (strncmp(line, "{\"device\": ", 11) != 0 || !json_str(line, "device", dev, sizeof dev)) continue;
            if (strcmp(dev, name) == 0) continue;
            std::string l(line);
            while (!l.empty() && (l.back() == '\n' || l.back() == '\r' || l.back() == ',')) l.pop_back();
            keep.push_back(l);
        }
        fclose(f);
    }
    for (int dt = 0; dt < 2; ++dt)
        for (int iv = 0; iv < 2; ++iv) {
            bool any = false;
            for (int k = 0; k < kK; ++k) any = any || ctx->tuned[dt][iv][k] > 0;
            if (!any) continue;
            char buf[1024];
            int n = snprintf(buf, sizeof buf, "{\"device\": \"%s\", \"dtype\": \"%s\", \"inv_var\": %d, \"class_pix\": [",
                             name, dt ? "bf16" : "f32", iv);
            for (int k = 0; k < kK; ++k) n += snprintf(buf + n, sizeof buf - n, "%s%d", k ? ", " : "", fse::kClassPix[k]);
            n += snprintf(buf + n, sizeof buf - n, "], \"warps_per_cta\": [");
            for (int k = 0; k < kK; ++k) n += snprintf(buf + n, sizeof buf - n, "%s%d", k ? ", " : "", ctx->tuned[dt][iv][k]);
            n += snprintf(buf + n, sizeof buf - n, "], \"warps_per_stamp\": [");
            for (int k = 0; k < kK; ++k) n += snprintf(buf + n, sizeof buf - n, "%s%d", k ? ", " : "", ctx->tuned_nw[dt][iv][k]);
            snprintf(buf + n, sizeof buf - n, "]}");
            keep.push_back(buf);
        }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return set_error(c, FSE_EINVAL, "cannot write %s", tmp.c_str());
    fprintf(f, "{\"format\": \"%s\", \"entries\": [\n", kTuneFormat);
    for (size_t i = 0; i < keep.size(); ++i) fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fprintf(f, "]}\n");
    const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
    if (!ok) return set_error(c, FSE_EINVAL, "cannot write %s", path);
    return FSE_OK;
}

int fse_tuning_read(const char* path, const char* device, int32_t* shapes) {
    if (!path || !device || !shapes) return -FSE_EINVAL;
    FILE* f = fopen(path, "r");
    if (!f) return -FSE_EINVAL;
    for (int i = 0; i < 2 * 2 * kK * 2; ++i) shapes[i] = -1;   // no entry
    char line[4096];
    bool format_ok = false;
    int applied = 0;
    while (fgets(line, sizeof line, f)) {
        char fmt[64];
        if (json_str(line, "format", fmt, sizeof fmt)) format_ok = strcmp(fmt, kTuneFormat) == 0;
        char dev[256], dts[16];
        if (!format_ok || strncmp(line, "{\"device\": ", 11) != 0 || !json_str(line, "device", dev, sizeof dev) ||
            strcmp(dev, device) != 0 || !json_str(line, "dtype", dts, sizeof dts))
            continue;
        long ivv[1], pix[kK], w[kK], nw[kK];
        if (json_ints(line, "inv_var", ivv, 1) != 1) {
            const char* p = strstr(line, "\"inv_var\": ");
            if (!p) continue;
            ivv[0] = strtol(p + 11, nullptr, 10);
        }
        const int dt = strcmp(dts, "bf16") == 0 ? 1 : (strcmp(dts, "f32") == 0 ? 0 : -1);
        const int iv = ivv[0] != 0;
        if (dt < 0 || json_ints(line, "class_pix", pix, kK) != kK || json_ints(line, "warps_per_cta", w, kK) != kK ||
            json_ints(line, "warps_per_stamp", nw, kK) != kK)
            continue;
        // the entry must be for this library's size classes, and every shape
        // one that fse_autotune could have chosen (0 keeps the library default)
        bool ok = true;
        for (int k = 0; k < kK && ok; ++k) {
            ok = pix[k] == fse::kClassPix[k];
            if (!ok || w[k] == 0) continue;
            const bool pow2 = (w[k] == 1 || w[k] == 2 || w[k] == 4 || w[k] == 8) &&
                              (nw[k] == 1 || nw[k] == 2 || nw[k] == 4 || nw[k] == 8);
            ok = pow2 && w[k] % nw[k] == 0 &&
                 fse::smem_per_group(fse::kClassPix[k], iv != 0, static_cast<int>(nw[k])) * (w[k] / nw[k]) <=
                     227 * 1024;
        }
        if (!ok) continue;
        for (int k = 0; k < kK; ++k) {
            int32_t* e = shapes + ((dt * 2 + iv) * kK + k) * 2;
            e[0] = static_cast<int32_t>(w[k]);
            e[1] = w[k] ? static_cast<int32_t>(nw[k]) : 0;
        }
        ++applied;
    }
    fclose(f);
    return applied;
}

int fse_tuning_load(fse_ctx* ctx, const char* path) {
    if (!ctx || !path) return FSE_EINVAL;
    char name[256];
    if (!device_name(ctx->device, name, sizeof name)) return set_error(ctx, FSE_ECUDA, "device properties");
    int32_t shapes[2 * 2 * kK * 2];
    const int applied = fse_tuning_read(path, name, shapes);
    if (applied < 0) return set_error(ctx, FSE_EINVAL, "cannot read %s", path);
    if (applied == 0) return set_error(ctx, FSE_EINVAL, "%s holds no launch shapes for %s", path, name);
    // settings absent from the file keep the context's shapes
    for (int dt = 0; dt < 2; ++dt)
        for (int iv = 0; iv < 2; ++iv) {
            const int32_t* e = shapes + (dt * 2 + iv) * kK * 2;
            if (e[0] < 0) continue;
            for (int k = 0; k < kK; ++k) {
                ctx->tuned[dt][iv][k] = e[2 * k];
                ctx->tuned_nw[dt][iv][k] = e[2 * k + 1];
            }
        }
    ++ctx->tune_version;
    return FSE_OK;
}

int fse_partition(const fse_stamp* idx, int64_t count, int32_t parts, int64_t* starts) {
    if (!starts || parts < 1 || count < 0 || (count > 0 && !idx)) return FSE_EINVAL;
    // prefix sums of the pixels; a stamp of invalid size weighs one pixel (the
    // estimator only flags it)
    double total = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t h = idx[i].h, w = idx[i].w;
        total += (h >= 1 && w >= 1 && h <= FSE_MAX_SIDE && w <= FSE_MAX_SIDE) ? static_cast<double>(h * w) : 1.0;
    }
    starts[0] = 0;
    double run = 0.0;
    int64_t i = 0;
    for (int32_t r = 1; r < parts; ++r) {
        // the first stamp whose start lies at or past r/parts of the pixels
        const double target = total * r / parts;
        while (i < count && run < target) {
            const int64_t h = idx[i].h, w = idx[i].w;
            run += (h >= 1 && w >= 1 && h <= FSE_MAX_SIDE && w <= FSE_MAX_SIDE) ? static_cast<double>(h * w) : 1.0;
            ++i;
        }
        starts[r] = i;
    }
    starts[parts] = count;
    return FSE_OK;
}

int fse_star_fit(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                 int64_t count, const fse_result* moments, int profile, const fse_opts* opts,
                 fse_star_result* out, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count < 0 || count > 0x7fffffffLL) return set_error(ctx, FSE_EINVAL, "count out of range");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    if (profile != FSE_STAR_GAUSS && profile != FSE_STAR_MOFFAT)
        return set_error(ctx, FSE_EINVAL, "unknown star profile %d", profile);
    fse_opts o;
    if (opts) o = *opts; else fse_opts_default(&o);
    int rc = check_opts(ctx, &o);
    if (rc) return rc;
    if (count == 0) return FSE_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    if (!pix || !idx || !moments || !out)
        return set_error(ctx, FSE_EINVAL, "pix, idx, moments and out must not be NULL");
    const void* dev_ptrs[] = {pix, idx, moments, out, scale};
    for (const void* q : dev_ptrs)
        if (q && !is_device_ptr(q))
            return set_error(ctx, FSE_EINVAL, "all array arguments must be device pointers");
    fse::StarArgs a;
    memset(&a, 0, sizeof a);
    a.pix = pix;
    a.dtype = dtype;
    a.scale = scale;
    a.idx = idx;
    a.count = count;
    a.moments = moments;
    a.out = out;
    a.profile = profile;
    a.max_pix = o.max_pix > 0 ? o.max_pix : FSE_MAX_PIX;
    a.tol = static_cast<float>(o.tol_sig);
    a.max_iter = o.max_iter_mom;
    a.queue = ctx->d_queue + (ctx->next_queue++ % kQueues);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "work counter reset");
    e = fse::launch_star(a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "star launch");
    return FSE_OK;
}

static int moment_grad(fse_ctx* ctx, bool jvp, const void* pix, int dtype, const float* scale,
                       const fse_stamp* idx, int64_t count, const fse_result* moments, int mode, const float* v,
                       float* dpix, const float* tangent, float* dtheta, uint32_t* status, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count < 0 || count > 0x7fffffffLL) return set_error(ctx, FSE_EINVAL, "count out of range");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    if (mode & ~(FSE_MOM_ELLIP | FSE_MOM_SIGW_FIXED | FSE_MOM_SIGW_R50))
        return set_error(ctx, FSE_EINVAL, "unknown mode bits 0x%x", mode);
    if ((mode & FSE_MOM_SIGW_FIXED) && (mode & FSE_MOM_SIGW_R50))
        return set_error(ctx, FSE_EINVAL, "FSE_MOM_SIGW_FIXED and FSE_MOM_SIGW_R50 exclude each other");
    if (count == 0) return FSE_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    const void* need[] = {pix, idx, moments, jvp ? static_cast<const void*>(tangent) : v,
                          jvp ? static_cast<const void*>(dtheta) : dpix};
    for (const void* q : need)
        if (!q) return set_error(ctx, FSE_EINVAL, "a required array argument is NULL");
    const void* dev_ptrs[] = {pix, idx, moments, v, dpix, tangent, dtheta, scale, status};
    for (const void* q : dev_ptrs)
        if (q && !is_device_ptr(q))
            return set_error(ctx, FSE_EINVAL, "all array arguments must be device pointers");
    fse::MomentGradArgs a;
    memset(&a, 0, sizeof a);
    a.pix = pix;
    a.dtype = dtype;
    a.scale = scale;
    a.idx = idx;
    a.count = count;
    a.moments = moments;
    a.mode = mode;
    a.v = v;
    a.dpix = dpix;
    a.tangent = tangent;
    a.dtheta = dtheta;
    a.status = status;
    if (!jvp) {
        // the analysis kernel's per-stamp coefficients for the write kernel
        const int rc = grow(ctx, &ctx->d_vjp, &ctx->vjp_cap, static_cast<size_t>(count));
        if (rc) return rc;
        a.coef = ctx->d_vjp;
    }
    if (!jvp && (mode & FSE_MOM_SIGW_R50)) {
        // the ring launch's growth-curve records for the analysis kernel
        const int rc = grow(ctx, &ctx->d_r50, &ctx->r50_cap, static_cast<size_t>(count));
        if (rc) return rc;
        a.r50g = ctx->d_r50;
    }
    a.queue = ctx->d_queue + (ctx->next_queue++ % kQueues);
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "work counter reset");
    e = fse::launch_moment_grad(a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "moment gradient launch");
    return FSE_OK;
}

int fse_moment_vjp(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                   int64_t count, const fse_result* moments, int mode, const float* v, float* dpix,
                   uint32_t* status, void* stream) {
    return moment_grad(ctx, false, pix, dtype, scale, idx, count, moments, mode, v, dpix, nullptr, nullptr,
                       status, stream);
}

int fse_moment_jvp(fse_ctx* ctx, const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                   int64_t count, const fse_result* moments, int mode, const float* tangent, float* dtheta,
                   uint32_t* status, void* stream) {
    return moment_grad(ctx, true, pix, dtype, scale, idx, count, moments, mode, nullptr, nullptr, tangent,
                       dtheta, status, stream);
}

int fse_cutout(fse_ctx* ctx, const void* images, int dtype, const float* scale, const fse_stamp* img_idx,
               int64_t count, double side_factor, int min_side, int max_side, fse_cutout_info* info,
               fse_stamp* out_idx, void* out_pix, int64_t out_capacity, int64_t* out_total, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count < 0) return set_error(ctx, FSE_EINVAL, "count out of range");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    if (!(side_factor > 0.0) || !std::isfinite(side_factor))
        return set_error(ctx, FSE_EINVAL, "side_factor must be positive and finite");
    if (min_side < 1 || max_side < min_side || max_side > 128)
        return set_error(ctx, FSE_EINVAL, "need 1 <= min_side <= max_side <= 128");
    if (out_capacity < 0) return set_error(ctx, FSE_EINVAL, "out_capacity must not be negative");
    if (count == 0) return FSE_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    if (!images || !img_idx || !info || !out_idx || !out_total)
        return set_error(ctx, FSE_EINVAL, "images, img_idx, info, out_idx and out_total must not be NULL");
    const void* dev_ptrs[] = {images, img_idx, info, out_idx, out_total, out_pix, scale};
    for (const void* q : dev_ptrs)
        if (q && !is_device_ptr(q))
            return set_error(ctx, FSE_EINVAL, "all array arguments must be device pointers");
    fse::CutoutArgs a;
    memset(&a, 0, sizeof a);
    a.images = images;
    a.dtype = dtype;
    a.scale = scale;
    a.img_idx = img_idx;
    a.count = count;
    a.side_factor = side_factor;
    a.min_side = min_side;
    a.max_side = max_side;
    a.info = info;
    a.out_idx = out_idx;
    a.out_pix = out_pix;
    a.out_capacity = out_capacity;
    a.out_total = out_total;
    cudaError_t e = fse::launch_cutout(a, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cut-out launch");
    return FSE_OK;
}

int fse_sersic_b(fse_ctx* ctx, const double* n, double* b, double* db, int64_t count, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count == 0) return FSE_OK;
    if (count < 0 || !n || !b) return set_error(ctx, FSE_EINVAL, "bad arguments");
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    if (!is_device_ptr(n) || !is_device_ptr(b) || (db && !is_device_ptr(db)))
        return set_error(ctx, FSE_EINVAL, "n, b and db must be device pointers");
    cudaError_t e = fse::eval_bn(n, b, db, count, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "b(n) evaluation");
    return FSE_OK;
}

int fse_sersic_chi2_grad(fse_ctx* ctx, const void* pix, int dtype, const float* scale,
                         const fse_stamp* idx, int64_t count, const float* inv_var,
                         const float* params, const double* gout, double* chi2, float* dparams,
                         float* dpix, void* stream) {
    if (!ctx) return FSE_EINVAL;
    if (count < 0 || count > 0x7fffffffLL) return set_error(ctx, FSE_EINVAL, "count out of range");
    if (dtype != FSE_F32 && dtype != FSE_BF16) return set_error(ctx, FSE_EINVAL, "unknown dtype %d", dtype);
    if (count == 0) return FSE_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return set_error(ctx, FSE_ECUDA, "cannot select device %d", ctx->device);
    if (!pix || !idx || !params) return set_error(ctx, FSE_EINVAL, "pix, idx and params must not be NULL");
    if (!chi2 && !dparams && !dpix) return set_error(ctx, FSE_EINVAL, "no output requested");
    const void* dev_ptrs[] = {pix, idx, params, scale, inv_var, gout, chi2, dparams, dpix};
    for (const void* q : dev_ptrs)
        if (q && !is_device_ptr(q))
            return set_error(ctx, FSE_EINVAL, "all array arguments must be device pointers");
    fse::GradArgs a;
    memset(&a, 0, sizeof a);
    a.pix = pix;
    a.dtype = dtype;
    a.scale = scale;
    a.idx = idx;
    a.count = count;
    a.inv_var = inv_var;
    a.params = params;
    a.gout = gout;
    a.chi2 = chi2;
    a.dparams = dparams;
    a.dpix = dpix;
    a.queue = ctx->d_queue + (ctx->next_queue++ % kQueues);
    a.bnf = fse::bn_table_f32();
    if (!a.bnf) return set_error(ctx, FSE_ECUDA, "b(n) table address");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "work counter reset");
    e = fse::launch_chi2_grad(a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "chi2/adjoint launch");
    return FSE_OK;
}

int fse_sync_check(fse_ctx* ctx, void* stream) {
    if (!ctx) return FSE_EINVAL;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronise");
    unsigned int flag = 0;
    e = cudaMemcpy(&flag, ctx->d_err, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word read");
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(unsigned int));
        return set_error(ctx, FSE_ETIMEOUT, "a bounded device wait expired");
    }
    return FSE_OK;
}

int fse_fit_batch_static(const void* pix, int dtype, const float* scale, const fse_stamp* idx,
                         int64_t count, const float* inv_var, const fse_opts* opts,
                         fse_result* out, void* stream, char* err, size_t err_len) {
    fse_ctx sink;   // on the stack: only the error text of the shared checks
    if (err && err_len) err[0] = 0;
    auto fail = [&](int rc) {
        if (err && err_len) snprintf(err, err_len, "%s", sink.err);
        return rc;
    };
    if (count > kStaticMaxCount)
        return fail(set_error(&sink, FSE_EINVAL,
                              "count %lld exceeds %lld, the largest batch the static work counter "
                              "can index", static_cast<long long>(count),
                              static_cast<long long>(kStaticMaxCount)));
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return fail(set_error(&sink, FSE_ECUDA, "no usable current CUDA device"));
    }
    sink.device = dev;
    fse::LaunchArgs a;
    int rc = prepare(&sink, pix, dtype, scale, idx, count, inv_var, opts, out, fse::kStageAll, &a);
    if (rc) return fail(rc);
    if (count == 0) return FSE_OK;
    unsigned int* scratch = nullptr;
    {
        // first call on this device: the b(n) table (static device storage,
        // built by a kernel, then a device synchronise) and the scratch address
        std::lock_guard<std::mutex> lk(g_table_mutex);
        e = ensure_bn_table(dev);
        if (e != cudaSuccess) return fail(cuda_fail(&sink, e, "b(n) table"));
        const unsigned long long cid = fse::current_context_id();
        if (!g_static_addr[dev] || g_static_ctx[dev] != cid) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return fail(cuda_fail(&sink, e, "static scratch address"));
            g_static_addr[dev] = static_cast<unsigned int*>(p);
            g_static_ctx[dev] = cid;
        }
        scratch = g_static_addr[dev];
    }
    a.queue = scratch;
    a.err = scratch + 1;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    // both words must start at zero: one stream-ordered clear before the launch
    e = cudaMemsetAsync(scratch, 0, kStaticWords * sizeof(unsigned int), s);
    if (e != cudaSuccess) return fail(cuda_fail(&sink, e, "static scratch clear"));
    e = fse::launch_estimator(a, s);
    if (e != cudaSuccess) return fail(cuda_fail(&sink, e, "estimator launch"));
    return FSE_OK;
}

}  // extern "C"
