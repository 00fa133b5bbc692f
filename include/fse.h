/*
 * fse.h -- C ABI of libfse, a GB300 (sm_103a) implementation of the fast
 * shape estimator of Li, Xin & Cui (2012), "Fast Shape Estimation for
 * Galaxies and Stars":
 *   1. centroid from Gaussian-weighted first moments with a fixed gain
 *      (Sec. 2, Eqs. 2-6);
 *   2. ellipticity from the KSB shear polarisability with an elliptical
 *      weight, iterated until the weight's ellipticity matches the object's
 *      (Sec. 3, Eqs. 7-9; Appendix A, Eqs. A1-A6; Appendix B, Eqs. B7-B14);
 *   3. a fit of the Sérsic profile (Eq. 10) over (r_e, n), with the amplitude
 *      I0 at its closed form (Eq. 13) and chi^2 as in Eq. 11 (Sec. 4.1),
 * applied to many postage stamps at once.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - A stamp is h x w pixels, row-major.  Pixel (row i, column j) has its
 *    centre at (x = j, y = i) in stamp coordinates.
 *  - Pixels of all stamps sit in one flat buffer; stamp s starts at element
 *    idx[s].offset.  Stamps may be unaligned, of different sizes, and in any
 *    order.  1 <= h, w <= FSE_MAX_SIDE and h*w <= opts->max_pix <=
 *    FSE_MAX_PIX; the estimator reports a stamp outside that range with
 *    FSE_ST_BAD_SIZE and does no other work on it.
 *  - Pixel type FSE_F32: float.  FSE_BF16: bfloat16, decoded as
 *    (float)pix * scale[s] with one float scale per stamp.
 *  - inv_var (optional, may be NULL): per-pixel 1/sigma_i^2 as float, laid out
 *    like the pixels; NULL means sigma_i = 1.  It weights chi^2 (Eq. 11) and
 *    the amplitude of Eq. 13; the moments do not use it.
 *  - Ellipticity g = (e1, e2) is the shear-type ellipticity of Eq. A1:
 *      R^2 = [(1-e1)^2+e2^2] dx^2 + [(1+e1)^2+e2^2] dy^2 - 4 e2 dx dy,
 *    the Sérsic radius is r = R / (1-|g|) (so r_e is the half-light radius
 *    along the major axis) and the axis ratio is q = (1-|g|)/(1+|g|).
 *  - Device entry points take DEVICE pointers owned by the caller (pix, scale,
 *    idx, inv_var, out) and a HOST pointer to the options (NULL = defaults).
 *    They are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream); out is complete when the stream reaches that point.
 *  - Return codes describe the call, never a stamp: FSE_OK, or FSE_EINVAL
 *    (bad argument; nothing launched), FSE_ENOMEM, FSE_ECUDA (a CUDA error;
 *    fse_last_error() gives the text), FSE_ETIMEOUT (a bounded device wait
 *    expired), FSE_EUNSUPPORTED.  Per-stamp problems go to fse_result.status.
 *    No call aborts, traps or prints.
 *  - count == 0 is a no-op returning FSE_OK.
 *  - One fse_ctx may be used from one host thread at a time; calls that
 *    overlap on the GPU must use different streams (up to 64 in flight).
 */
#ifndef FSE_H
#define FSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSE_OK            0
#define FSE_EINVAL        1
#define FSE_ENOMEM        2
#define FSE_ECUDA         3
#define FSE_ETIMEOUT      4
#define FSE_EUNSUPPORTED  5

#define FSE_MAX_PIX       (128 * 128)
#define FSE_MAX_SIDE      128

/* fse_result.status bits */
#define FSE_ST_MOM_CONVERGED  (1u << 0)  /* centroid/ellipticity reached the stop rule      */
#define FSE_ST_FIT_CONVERGED  (1u << 1)  /* profile fit reached its stop rule               */
#define FSE_ST_MOM_MAXITER    (1u << 2)  /* moment loop hit max_iter_mom                    */
#define FSE_ST_FIT_MAXITER    (1u << 3)  /* fit hit max_iter_fit                            */
#define FSE_ST_NONFINITE      (1u << 4)  /* a NaN/Inf pixel: stamp skipped                  */
#define FSE_ST_BAD_SIZE       (1u << 5)  /* h*w outside [1, max_pix]: stamp skipped         */
#define FSE_ST_MOM_FAILED     (1u << 6)  /* sum I W <= 0, T <= 0, |g| >= 0.95, centre left
                                            the stamp or P^SH singular: no fit              */
#define FSE_ST_FIT_BOUND      (1u << 7)  /* r_e or n ended on a bound                       */
#define FSE_ST_FIT_SINGULAR   (1u << 8)  /* damped normal equations singular                */
#define FSE_ST_NONPOS_FLUX    (1u << 9)  /* fitted I0 <= 0                                   */
#define FSE_ST_SIGW_CLAMPED   (1u << 10) /* sigma_w clamped to [0.5, min(h,w)/2]            */
#define FSE_ST_INIT_FALLBACK  (1u << 11) /* stamp total <= 0: sigma_w from r50 = 1.1774 px  */
#define FSE_ST_TIMEOUT        (1u << 12) /* a bounded device wait expired for this stamp    */
#define FSE_ST_MOM_REFINE2    (1u << 13) /* informational: a second moment refinement ran    */
#define FSE_ST_FIT_REFINE2    (1u << 14) /* informational: a second fit refinement ran       */
#define FSE_ST_NO_ROOM        (1u << 15) /* fse_cutout: the output buffer had no room for it */

/* fse_opts.flags: fse_fit_batch_ragged captures its launch sequence into a
 * CUDA graph on first use and replays it while its arguments are unchanged. */
#define FSE_FLAG_GRAPH        (1u << 0)

/* Star profiles of Sec. 4.2 (fse_star_fit). */
#define FSE_STAR_GAUSS        0
#define FSE_STAR_MOFFAT       1

/* Implicit gradients of the moment fixed point (fse_moment_vjp / _jvp). */
#define FSE_MOM_ELLIP         1   /* g1, g2 are parameters (Secs. 2-3); else g = 0 (Sec. 2)  */
#define FSE_MOM_SIGW_FIXED    2   /* sigma_w held                                           */
#define FSE_MOM_SIGW_R50      4   /* sigma_w = r50/sqrt(2 ln 2) of the start-up growth curve */

typedef struct fse_ctx fse_ctx;

/* Stamp index entry (16 bytes).  offset counts elements (not bytes). */
typedef struct {
    int64_t offset;
    int32_t h;
    int32_t w;
} fse_stamp;

enum { FSE_F32 = 0, FSE_BF16 = 1 };

/* Options (host struct; fse_opts_default fills the defaults below). */
typedef struct {
    size_t  size;           /* sizeof(fse_opts), for versioning                         */
    double  tol_pos;        /* stop when |centroid step| <= tol_pos px        (1e-6)    */
    double  tol_g;          /* ... and |ellipticity step| <= tol_g            (1e-6)    */
    double  tol_sig;        /* ... and |sigma_w step|/sigma_w <= tol_sig, mode 0 (1e-6) */
    double  tol_fit;        /* fit stops when max relative (r_e, n) step <= tol_fit (1e-4) */
    int32_t max_iter_mom;   /* moment iterations                              (60)      */
    int32_t max_iter_fit;   /* fit iterations                                 (60)      */
    double  k_gain;         /* centroid gain k of Sec. 2.  0 (default): k determined
                               from the current moments (a Newton step) near the fixed
                               point, 0.75 elsewhere; > 0: that fixed gain (the paper's
                               0.75).  The fixed point does not depend on k.    (0)     */
    int32_t sigw_mode;      /* 1: sigma_w = r50/sqrt(2 ln 2) fixed; 0: matched-weight
                               rule sigma_w^2 = sum I W R^2 / sum I W (Sec. 4.2.1)  (1)  */
    int32_t max_pix;        /* upper bound of h*w over the batch; sets the shared-memory
                               tile (0 = FSE_MAX_PIX)                         (0)       */
    double  n_min, n_max;   /* bounds on n                                    (0.2, 10) */
    double  re_min;         /* lower bound on r_e, px                         (0.2)     */
    double  re_max_frac;    /* upper bound on r_e = re_max_frac * max(h, w)   (2)       */
    double  lm_lambda0;     /* initial Levenberg-Marquardt damping            (1e-3)    */
    uint32_t flags;         /* FSE_FLAG_* bits                                 (0)       */
    int32_t warps_per_cta;  /* launch shape: 0 (library choice), 1, 2, 4 or 8                      */
    int32_t warps_per_stamp;/* warps sharing one stamp (whole chain only): 0 (library
                               choice: 1 up to 48x48 tiles, then 2, 4, 8 up to 128x128),
                               1, 2, 4 or 8; warps_per_cta must be a multiple     (0)  */
    int32_t supersample;    /* S in [1, 8]: the fit's Sersic model of a pixel is the mean
                               of S x S point samples on a regular sub-grid, the pixel
                               integral to O(1/S^2) (pixelation, Sec. 4.2); 0 or 1: the
                               pixel centre (Sec. 4.1).  S > 1 runs one warp per stamp
                               and costs about S^2 times the fit.              (1)       */
} fse_opts;

/* Per-stamp result (64 bytes). */
typedef struct {
    float    x0, y0;        /* centroid, stamp pixel coordinates                        */
    float    e1, e2;        /* ellipticity g                                            */
    float    I0;            /* central intensity, Eq. 13 at the optimum                 */
    float    re;            /* half-light radius along the major axis, px               */
    float    n;             /* Sérsic index                                              */
    float    flux;          /* 2 pi n Gamma(2n) b^-2n I0 r_e^2 q                        */
    double   chi2;          /* Eq. 11 at the optimum                                     */
    int32_t  npix;          /* h*w                                                      */
    int32_t  it_mom;        /* moment iterations (weighted passes)                      */
    int32_t  it_fit;        /* fit passes: profile evaluations after the start pass     */
    uint32_t status;        /* FSE_ST_* bits                                            */
    float    sigma_w;       /* weight size used by the moments, px                      */
    float    r50;           /* growth-curve half-light radius of the start-up, px       */
} fse_result;

/* Star profile result (32 bytes), fse_star_fit. */
typedef struct {
    float    size;          /* Gaussian sigma or Moffat r_d along the major axis, px   */
    float    beta;          /* Moffat beta (0 for the Gaussian)                         */
    float    I0;            /* central intensity                                        */
    float    flux;          /* Gaussian 2 pi s^2 I0 q; Moffat pi r_d^2 I0 q / (beta-1)  */
    float    r50;           /* half-light radius along the major axis, px               */
    int32_t  iters;         /* weight-size iterations                                   */
    uint32_t status;        /* FSE_ST_MOM_CONVERGED / _MAXITER / _FAILED, BAD_SIZE, ... */
    float    reserved;
} fse_star_result;

/* One cut-out of fse_cutout (24 bytes). */
typedef struct {
    int32_t  row0, col0;    /* first row and column of the square in its image        */
    int32_t  h, w;          /* its size after cutting to the image (0 if refused)     */
    float    r50;           /* growth-curve half-light radius around the brightest px */
    uint32_t status;        /* 0, FSE_ST_NONFINITE, FSE_ST_BAD_SIZE, FSE_ST_INIT_FALLBACK,
                               FSE_ST_NO_ROOM                                          */
} fse_cutout_info;

/* Create a context on CUDA device `device`: selects the device, builds the
 * device table of the Sérsic b(n) (root of P(2n, b) = 1/2, Eq. 10) and b'(n),
 * and allocates a small workspace.  *ctx is NULL on failure. */
int fse_create(fse_ctx **ctx, int device);

/* Release the context and its device memory (synchronises the device). */
void fse_destroy(fse_ctx *ctx);

/* Text of the last error of this context ("" if none).  Owned by ctx. */
const char *fse_last_error(const fse_ctx *ctx);

/* Defaults listed in fse_opts. */
void fse_opts_default(fse_opts *opts);

/* Sec. 2 alone (Eqs. 2-6): per stamp, start at the brightest pixel (ties: the
 * lowest row-major index), take sigma_w from the growth-curve half-light
 * radius r50 around it (Sec. 4.1), and iterate x_c += <x>/(k N) with a
 * circular Gaussian weight to the stop rule.  Writes x0, y0, sigma_w, r50,
 * npix, it_mom, status; zeroes the other fields of out[s]. */
int fse_centroid(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                 const fse_stamp *idx, int64_t count, const float *inv_var,
                 const fse_opts *opts, fse_result *out, void *stream);

/* Secs. 2-3 together (Eqs. 5-9, A1-A6, B7-B14): from out[s].x0, y0 and
 * sigma_w, iterate the centroid step and the ellipticity step
 * dg = (1-|g_w|^2) (P^SH)^-1 (e^obs - e_w), starting from g_w = 0 (the
 * circular-weight KSB estimate), to the stop rule.  Reads and rewrites
 * x0, y0 and sigma_w; writes e1, e2, it_mom and the moment status bits. */
int fse_ellipticity(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                    const fse_stamp *idx, int64_t count, const float *inv_var,
                    const fse_opts *opts, fse_result *inout, void *stream);

/* Sec. 4.1 fit (Eqs. 10-13) with centre and ellipticity held at out[s].x0,
 * y0, e1, e2: start at r_e = 1.1774 sigma_w / (1-|g|) and the best n of
 * {0.5, 1, 2, 4}, then Levenberg-Marquardt over (r_e, n) with I0 at its
 * closed form.  Writes I0, re, n, flux, chi2, it_fit and the fit status bits. */
int fse_sersic_fit(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                   const fse_stamp *idx, int64_t count, const float *inv_var,
                   const fse_opts *opts, fse_result *inout, void *stream);

/* The whole chain of Sec. 4.1 (start-up, centroid + ellipticity from the
 * brightest pixel, fit) in three persistent launches on `stream`: the start-up
 * (brightest pixel, growth-curve r50, sigma_w), the moment iteration, then the
 * fit of every stamp whose moments converged.  Results are those of the three
 * single stages run in turn. */
int fse_fit_batch(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                  const fse_stamp *idx, int64_t count, const float *inv_var,
                  const fse_opts *opts, fse_result *out, void *stream);

/* The same chain launched per stamp (one warp per launch, three launches per
 * stamp).  A baseline for measurement only; results are identical to
 * fse_fit_batch. */
int fse_fit_batch_plain(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                        const fse_stamp *idx, int64_t count, const float *inv_var,
                        const fse_opts *opts, fse_result *out, void *stream);

/* fse_fit_batch on HOST buffers: pix (npix_total elements of dtype), scale
 * (count floats or NULL), idx, inv_var (or NULL) and out are host pointers
 * (page-locked memory lets the copies overlap the kernels).  The call copies
 * the inputs to context-owned device buffers in chunks (from 8192 stamps up,
 * 9 chunks of 2, 4, 6, 8, 10, 10, 10, 8 and 6 64ths of the batch, else one)
 * on a context copy stream,
 * runs each chunk's chain on `stream` or a second context stream as soon as
 * its copy is done, copies the results back and returns when out[] is
 * complete.  npix_total bounds every idx[s].offset + h*w; a stamp outside it
 * returns FSE_EINVAL before any kernel runs, with out[] untouched (each chunk
 * is checked just before its copy, so the chunks before it may already have
 * been copied into the context's buffers).  Results equal those of
 * fse_fit_batch byte for byte.  One host-buffer call at a time per context
 * (the device buffers and events are the context's). */
int fse_fit_batch_host(fse_ctx *ctx, const void *pix, int64_t npix_total, int dtype,
                       const float *scale, const fse_stamp *idx, int64_t count,
                       const float *inv_var, const fse_opts *opts, fse_result *out,
                       void *stream);

/* fse_fit_batch for a RAGGED batch (stamps of different sizes, 1 to
 * FSE_MAX_PIX pixels, in any order).  The stamps are bucketed on the device
 * into seven size classes (h*w up to 16^2, 24^2, 32^2, 48^2, 64^2, 96^2,
 * 128^2), and each class runs in its own pair of persistent launches whose
 * shared-memory tile fits that class, largest class first.  Results are those of
 * fse_fit_batch, stamp by stamp.  opts->max_pix is not used (each class sets
 * its own); opts->warps_per_cta, if non-zero, applies to every class, else
 * the class uses the choice of fse_autotune or the library default.  With
 * FSE_FLAG_GRAPH in opts->flags the classification and the class launches are
 * captured into a CUDA graph on a context stream the first time, and later
 * calls with the same pointers, count, options and tuning replay it on
 * `stream`.  Device workspace: 4 bytes per stamp, grown as needed (a grown
 * buffer is a new pointer, so the next call captures again).  One ragged call
 * may be in flight per context. */
int fse_fit_batch_ragged(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                         const fse_stamp *idx, int64_t count, const float *inv_var,
                         const fse_opts *opts, fse_result *out, void *stream);

/* Choose the launch shape of each size class of fse_fit_batch_ragged -- warps
 * per stamp (1, 2, 4, 8) and stamp groups per CTA, at most 8 warps per CTA and
 * as far as shared memory allows -- by timing the class launches on this
 * batch (each candidate twice, the faster counts).  The choice is kept
 * in the context for this dtype and inverse-variance setting and used by
 * later ragged calls.  out receives the batch's results.  Synchronises
 * `stream`.  No counterpart in the paper: a launch-shape search. */
int fse_autotune(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                 const fse_stamp *idx, int64_t count, const float *inv_var,
                 const fse_opts *opts, fse_result *out, void *stream);

/* Keep the launch shapes fse_autotune chose for this context's device, so that
 * a later process can reuse them instead of timing again (no counterpart in the
 * paper).  fse_tuning_save writes every dtype and inverse-variance setting
 * tuned so far to the JSON file `path` (written to path.tmp, then renamed), one
 * entry per device name, dtype and setting, each with the size classes' pixel
 * bounds, warps per CTA and warps per stamp; entries of other devices already
 * in the file are kept.  fse_tuning_load applies the entries for this
 * context's device name whose size classes match this library's and whose
 * shapes are valid ones (1, 2, 4 or 8 warps, a multiple of the warps per
 * stamp, within shared memory), as if fse_autotune had chosen them; a CUDA
 * graph cached by fse_fit_batch_ragged is captured again.  Returns FSE_OK, or
 * FSE_EINVAL (NULL argument, unreadable or unwritable file, no applicable
 * entry: the context keeps its shapes).  Host calls; no device work. */
int fse_tuning_save(const fse_ctx *ctx, const char *path);
int fse_tuning_load(fse_ctx *ctx, const char *path);

/* The launch shapes a file written by fse_tuning_save holds for the device
 * named `device` (cudaDeviceProp.name), read without a context or a GPU, with
 * the checks fse_tuning_load applies (format "libfse-launch-shapes/1", this
 * library's size classes, valid shapes; other entries are skipped).  shapes
 * (host, 56 int32) receives, at ((dtype * 2 + inv_var) * 7 + class) * 2, the
 * warps per CTA and the warps per stamp (0, 0 for the library default), or
 * -1, -1 for a dtype and inverse-variance setting the file has no entry for.
 * Returns the number of entries read (0 or more), or -FSE_EINVAL for a NULL
 * argument or a file that cannot be opened.  Host call. */
int fse_tuning_read(const char *path, const char *device, int32_t *shapes);

/* The launch shape the ragged path uses for each of the seven size classes
 * (tuned or default), for a dtype and with (1) or without (0) inverse
 * variance: warps per CTA and warps per stamp (host arrays of 7; the second
 * may be NULL). */
int fse_tuned_warps(const fse_ctx *ctx, int dtype, int has_inv_var, int32_t *warps_per_cta,
                    int32_t *warps_per_stamp);

/* Star profiles of Sec. 4.2 from weighted radial moments, at the centre and
 * ellipticity of moments[s] (x0, y0, e1, e2 and sigma_w of a converged moment
 * stage: fse_ellipticity or fse_fit_batch).  r is the semi-major-axis radius
 * R(g)/(1-|g|); the pixel sums r_k = sum I W r^k carry the axis ratio
 * q = (1-|g|)/(1+|g|), which cancels from every ratio.
 *   FSE_STAR_GAUSS: W = exp(-r^2/2 s_w^2), sigma = sqrt(r2/r0), s_w <- sigma to
 *     its fixed point (started at sigma_w/(1-|g|)), I0 = r0/(pi sigma^2 q).
 *   FSE_STAR_MOFFAT: W = (1 + r^2/r_dw^2)^-3, beta = 1/(r4 r0/(2 r2^2) - 1),
 *     r_d = sqrt(r2/r0 (beta+1)), r_dw <- r_d (started at 2.35 sigma_w/(1-|g|)),
 *     I0 = r0 (beta+2)/(pi r_d^2 q).
 * The iteration stops at a relative size step of opts->tol_sig within
 * opts->max_iter_mom passes; opts->max_pix sizes the shared-memory tile.
 * A stamp whose moments did not converge gets FSE_ST_MOM_FAILED.  The sums are
 * over pixel centres (no pixel integration), so small stars carry the
 * pixelation bias the paper reports.  Device pointers; asynchronous. */
int fse_star_fit(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                 const fse_stamp *idx, int64_t count, const fse_result *moments, int profile,
                 const fse_opts *opts, fse_star_result *out, void *stream);

/* Implicit-function derivatives of the moment fixed point (Secs. 2-3) with
 * respect to the pixels.  The moment stage stops at theta = (x0, y0, e1, e2,
 * sigma_w) where its steps vanish: with t = pixel - centre, R^2 of Eq. A1,
 * W = exp(-R^2 / 2 sigma_w^2) and e_w = 2g/(1+g^2),
 *   F_k = sum_p I_p W m_k(t) = 0,  m = (t1, t2, (t1^2 - t2^2) - e_w1 (t1^2 + t2^2),
 *                                      2 t1 t2 - e_w2 (t1^2 + t2^2), R^2 - sigma_w^2)
 * (zero centroid step, Eqs. 3-6; e^obs = e_w, the zero of the step of Eq. 9;
 * the matched weight).  Hence d theta / d I_p = -J^-1 W(p) m(p) with
 * J = dF/dtheta.  mode: FSE_MOM_ELLIP for the Secs. 2-3 fixed point (without
 * it g = 0 is held: the Sec. 2 centroid stage), and the sigma_w rule the moment
 * stage used, which the caller must name: FSE_MOM_SIGW_R50 for moments
 * computed with fse_opts.sigw_mode = 1 (the fse_opts_default setting: sigma_w =
 * r50/sqrt(2 ln 2) from the start-up growth curve, Sec. 4.1, differentiated
 * with the brightest pixel and the crossing ring held); neither sigma_w bit for
 * sigw_mode = 0 (the matched weight); FSE_MOM_SIGW_FIXED to hold sigma_w.  A
 * stamp whose status has FSE_ST_SIGW_CLAMPED holds sigma_w.
 * moments[s]: x0, y0, e1, e2, sigma_w, r50 and status of a moment stage
 * (fse_centroid, fse_ellipticity or fse_fit_batch).
 * fse_moment_vjp: v[s*5 + k] = dL/dtheta_k (entries of held parameters are
 * ignored); writes dL/dI to dpix (fp32, at the element offsets of pix).
 * fse_moment_jvp: tangent (fp32, offsets of pix) = dI; writes dtheta[s*5 + k].
 * status[s] (optional): 0, or FSE_ST_MOM_FAILED (moments not converged),
 * FSE_ST_NONFINITE, FSE_ST_BAD_SIZE (h*w above FSE_MAX_PIX: nothing written),
 * FSE_ST_FIT_SINGULAR (J singular); such stamps get zero derivatives.
 * bf16 pixels are decoded with scale[s]; the derivatives are with respect to
 * the decoded intensities.  Device pointers; asynchronous on `stream`.  The
 * VJP runs up to three launches: with FSE_MOM_SIGW_R50 one for the growth
 * curve (a 48-byte record per stamp), one per stamp for the sums, J and the
 * solve (96 bytes of coefficients per stamp), then one that writes dL/dI from
 * them.  The records and coefficients live in grow-only scratch buffers of the
 * context, allocated, with a device synchronisation, when a call has more
 * stamps than any before (so not under stream capture); VJP calls on one
 * context that overlap on the GPU share them. */
int fse_moment_vjp(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                   const fse_stamp *idx, int64_t count, const fse_result *moments, int mode,
                   const float *v, float *dpix, uint32_t *status, void *stream);
int fse_moment_jvp(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                   const fse_stamp *idx, int64_t count, const fse_result *moments, int mode,
                   const float *tangent, float *dtheta, uint32_t *status, void *stream);

/* The cut-out of Sec. 4.1.  For each image s (img_idx[s] in `images`, fp32,
 * or bf16 decoded with scale[s] for the growth curve), r50 comes from the
 * growth curve around the brightest pixel (ties: lowest row-major index):
 * pixels summed in rings of integer radius (k-1 < d <= k) until half the
 * total, linear inside the crossing ring, in exact 64-bit fixed point.  The
 * square of side floor(side_factor * r50 + 0.5), clamped to [min_side,
 * max_side], starts side/2 (integer division) rows and columns before the
 * brightest pixel and is cut to the image.  The cut-outs are copied back to
 * back into out_pix (same dtype as the images; a bf16 cut-out keeps its
 * image's scale), in image order; out_idx[s] gets their offset and size and
 * info[s] the square and r50.  *out_total (device int64) receives the
 * elements of all cut-outs; with out_pix NULL only sizes and offsets are
 * written, so a first call can size the buffer.  A cut-out that does not fit
 * in out_capacity elements gets FSE_ST_NO_ROOM and is not copied.  Images of
 * more than 2^28 pixels get FSE_ST_BAD_SIZE; a crossing beyond a radius of
 * 2047 px gives r50 = NaN and the largest side.  1 <= min_side <= max_side
 * <= 128 (the largest stamp the estimator takes); side_factor > 0 (6 in the
 * paper).  Device pointers; asynchronous on `stream`. */
int fse_cutout(fse_ctx *ctx, const void *images, int dtype, const float *scale,
               const fse_stamp *img_idx, int64_t count, double side_factor, int min_side, int max_side,
               fse_cutout_info *info, fse_stamp *out_idx, void *out_pix, int64_t out_capacity,
               int64_t *out_total, void *stream);

/* Evaluate the device b(n) table (Eq. 10: P(2n, b) = 1/2) and its derivative
 * at count values n[i] in [0.2, 10] (device pointers, doubles).  For tests. */
int fse_sersic_b(fse_ctx *ctx, const double *n, double *b, double *db, int64_t count,
                 void *stream);

/* chi^2 (Eq. 11) of the elliptical Sérsic model (Eq. 10) at given parameters,
 * and its gradient (the adjoint) with respect to the parameters and to the
 * pixels.  params[s*7 + k] holds (x0, y0, e1, e2, I0, r_e, n) for stamp s, in
 * the conventions above (centre in stamp pixels, g of Eq. A1, r_e along the
 * major axis).  With residuals r_i = m_i - I_i and weights w_i (inv_var, or 1):
 *   chi2[s]            = sum_i w_i r_i^2                       (fp64)
 *   dparams[s*7 + k]   = gout[s] * 2 sum_i w_i r_i dm_i/dp_k    (fp32)
 *   dpix[offset_s + i] = gout[s] * (-2 w_i r_i)                 (fp32)
 * gout (count doubles, or NULL = 1 for every stamp) makes the call a
 * vector-Jacobian product.  dpix has the element layout of pix (each stamp at
 * its own offset) and is the derivative with respect to the decoded pixel
 * value; it is always fp32.  chi2, dparams and dpix may each be NULL (not
 * computed), but not all three.  The pixel at R^2 = 0 adds no derivative with
 * respect to the centre or the ellipticity, and d|g|/dg is taken as 0 at
 * g = 0.  A stamp whose size is outside [1, FSE_MAX_PIX], or whose parameters
 * are not finite or lie outside r_e > 0, |g| < 1, n in [0.129, 10.27] (the
 * b(n) table), gets NaN in chi2, dparams and (for a valid size) dpix.  All
 * arrays are device pointers; asynchronous on `stream`. */
int fse_sersic_chi2_grad(fse_ctx *ctx, const void *pix, int dtype, const float *scale,
                         const fse_stamp *idx, int64_t count, const float *inv_var,
                         const float *params, const double *gout, double *chi2,
                         float *dparams, float *dpix, void *stream);

/* Replicas over stamp ranges: the stamps are independent, so a batch spread
 * over several devices (or processes) is cut into `parts` contiguous index
 * ranges of about equal total pixels, each device runs fse_fit_batch on its
 * range, and the results are concatenated in range order (no collective on
 * the data path).  starts (host, parts + 1 entries) receives the boundaries:
 * range r is idx[starts[r] .. starts[r+1]), starts[0] = 0, starts[parts] =
 * count; range r starts at the first stamp at or past r/parts of the pixels,
 * so a range holds at most one stamp's pixels more than an equal share.  A
 * stamp of invalid size counts as one pixel.  idx is a HOST array.  Returns
 * FSE_OK, or FSE_EINVAL (NULL pointer, parts < 1, count < 0).  No counterpart
 * in the paper, which measured one galaxy at a time. */
int fse_partition(const fse_stamp *idx, int64_t count, int32_t parts, int64_t *starts);

/* Wait for `stream` and report a bounded device wait that expired during any
 * earlier call of this context (FSE_ETIMEOUT), or FSE_OK.  Clears the flag. */
int fse_sync_check(fse_ctx *ctx, void *stream);

/* fse_fit_batch without a context and without allocating device memory (the
 * paper has no counterpart: it concerns the library, not the method).  For
 * callers that cannot allocate at the point of the call, e.g. a service whose
 * device footprint is fixed after start-up, or code under a caching allocator
 * that owns all device memory.  Same arguments, layout and results as
 * fse_fit_batch, on the CURRENT CUDA device; all pointers but opts and err are
 * device pointers owned by the caller.
 *  - Scratch: a file-scope device array of two 32-bit words (the work counter
 *    and the error word), cleared by a cudaMemsetAsync on `stream` before each
 *    launch.  count is limited to 2^31 - 1 stamps, the range the counter
 *    indexes; a larger count returns FSE_EINVAL with a message.
 *  - First call on a device: builds the b(n) table (a kernel and a device
 *    synchronise) and looks up the scratch address; make it before any stream
 *    capture.  Later calls only clear the scratch and launch.  Both belong to
 *    the device's CUDA context: the first call after a cudaDeviceReset (a new
 *    primary context) sets them up again in the same way.
 *  - Calls that can overlap on the GPU (different streams or host threads)
 *    share the scratch and race: issue them in order on one stream.
 *  - A bounded device wait that expires marks the stamp FSE_ST_TIMEOUT.
 *  - err (may be NULL): on failure, a NUL-terminated message of at most
 *    err_len bytes; empty on success. */
int fse_fit_batch_static(const void *pix, int dtype, const float *scale, const fse_stamp *idx,
                         int64_t count, const float *inv_var, const fse_opts *opts,
                         fse_result *out, void *stream, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* FSE_H */
