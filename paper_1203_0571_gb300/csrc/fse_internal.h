// Internal interface between the C ABI layer (fse_api.cu) and the kernels
// (fse_kernels.cu).  Not installed; the public interface is include/fse.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fse.h"

namespace fse {

// Which part of the chain a launch runs.
enum Stage : int {
    kStageCentroid = 1,     // start-up + Sec. 2 centroid (circular weight)
    kStageEllipticity = 2,  // Secs. 2-3 from a given centre and sigma_w
    kStageFit = 3,          // Sec. 4.1 fit with centre and g fixed
    kStageAll = 4,          // whole chain: kStageStartup, kStageMoments, then kStageFit with chain_fit
    kStageMoments = 5,      // Secs. 2-3 from the start-up's record (the second launch of the chain)
    kStageStartup = 6,      // start-up alone: brightest pixel, growth-curve r50, sigma_w (Sec. 4.1);
                            // the first launch of the chain and of fse_centroid
};

// Options as the kernels see them (fp32 where the per-pixel code uses them).
struct DevOpts {
    float tol_pos, tol_g, tol_sig, tol_fit;
    int max_iter_mom, max_iter_fit;
    float k_gain;
    int sigw_mode;
    int max_pix;
    float n_min, n_max, re_min, re_max_frac;
    float lm_lambda0;
    int supersample;     // S > 1: the fit's model is the mean of S x S samples per pixel
    int ring_slots;      // rings of the start-up histogram a stamp of max_pix pixels can need
                         // (set at launch from max_pix)
};

struct LaunchArgs {
    const void* pix;
    int dtype;
    const float* scale;
    const fse_stamp* idx;
    int64_t count;
    const float* inv_var;
    fse_result* out;
    unsigned int* queue;     // persistent-kernel work counter (zeroed before launch)
    unsigned int* err;       // sticky error word (bounded waits that expired)
    DevOpts opts;
    int stage;
    int warps_per_cta;       // a multiple of warps_per_stamp
    int warps_per_stamp;     // 1, 2, 4 or 8 warps share a stamp (whole chain only)
    int num_ctas;            // 0 = library choice
    int static_assign;       // 1: warp w of the grid takes stamp w only (no counter)
    int chain_fit;           // kStageFit as the second launch of the chain: keeps every
                             // status bit of the record and fits only converged moments
    // Size-class launches of the ragged path: the launch takes the stamps
    // perm[range[0] .. range[0] + range[1]) (range in device memory, written by
    // the classification kernels earlier on the stream).  NULL: stamps 0..count.
    const int32_t* perm;
    const unsigned int* range;
};

// Size classes of the ragged path: class k holds the stamps with
// kClassPix[k-1] < h*w <= kClassPix[k] (stamps of invalid size go to class 0,
// where the kernel flags them without reading pixels).
constexpr int kClasses = 7;
constexpr int kClassPix[kClasses] = {16 * 16, 24 * 24, 32 * 32, 48 * 48, 64 * 64, 96 * 96, 128 * 128};

// Buckets count stamps into the size classes: counts/range/cursor are device
// arrays of kClasses, kClasses x 2 and kClasses unsigned ints; perm gets count
// stamp ids grouped by class.  counts must be zero on entry.
cudaError_t classify_stamps(const fse_stamp* idx, int64_t count, unsigned int* counts,
                            unsigned int* range, unsigned int* cursor, int32_t* perm,
                            cudaStream_t stream);

// Arguments of the chi^2 / adjoint kernel (fse_sersic_chi2_grad).
struct GradArgs {
    const void* pix;
    int dtype;
    const float* scale;
    const fse_stamp* idx;
    int64_t count;
    const float* inv_var;
    const float* params;     // count x 7: x0, y0, e1, e2, I0, r_e, n
    const double* gout;      // count upstream gradients, or NULL (= 1)
    double* chi2;            // count, or NULL
    float* dparams;          // count x 7, or NULL
    float* dpix;             // laid out like pix (fp32), or NULL
    unsigned int* queue;     // work counter (zeroed before launch)
    const float2* bnf;       // the device's fp32 b(n), b'(n) table (bn_table_f32)
};

// Arguments of the star-profile kernel (fse_star_fit, Sec. 4.2).
struct StarArgs {
    const void* pix;
    int dtype;
    const float* scale;
    const fse_stamp* idx;
    int64_t count;
    const fse_result* moments;   // centre, ellipticity and sigma_w of each stamp
    fse_star_result* out;
    int profile;                 // FSE_STAR_GAUSS or FSE_STAR_MOFFAT
    int max_pix;                 // shared-memory tile (pixels per warp)
    float tol;                   // relative step of the weight size that stops
    int max_iter;
    unsigned int* queue;         // work counter (zeroed before launch)
};

// Arguments of the implicit-gradient kernel of the moment fixed point
// (fse_moment_vjp / fse_moment_jvp).
// The growth curve of the start-up (Sec. 4.1) around the brightest pixel, for
// d sigma_w / d I: the crossing ring k (the first whose enclosed sum reaches
// half the total) and the constants of d sigma_w / d I_p in the three regions
// d <= k-1, k-1 < d <= k and d > k; for the JVP the tangent's sums over the
// two discs.  Written per stamp by the ring launch of the moment gradient.
struct R50Grad {
    int on;                  // sigma_w depends on the pixels
    int pr, pc, k;
    float c_in, c_ring, c_out;
    float u_in, u_disc;      // JVP: tangent summed over d <= k-1 and d <= k
    float pad[3];            // 48 bytes
};

// Per-stamp coefficients of the VJP's pixel gradient, dL/dI_p =
// -W(p) (c0 + c1 t1 + c2 t2 + c3 t1^2 + c4 t1 t2 + c5 t2^2) + the growth
// curve's ring term, written by the analysis kernel for the write kernel.
struct VjpCoef {
    float x0, y0, A, B, G4, cw;   // the weight at the fixed point
    float c[6];
    float kc_in, kc_ring, kc_out; // kappa d sigma_w / d I_p inside, on and outside the crossing ring
    float pc, pr, km2, k2;        // brightest pixel; (k-1)^2 (or -1) and k^2 of the crossing ring
    int ring, ok;
    float pad[3];                 // 96 bytes
};

struct MomentGradArgs {
    const void* pix;
    int dtype;
    const float* scale;
    const fse_stamp* idx;
    int64_t count;
    const fse_result* moments;   // theta = (x0, y0, e1, e2, sigma_w), status, r50
    int mode;                    // FSE_MOM_* bits
    const float* v;              // VJP: count x 5 upstream gradients
    float* dpix;                 // VJP: laid out like pix (fp32)
    const float* tangent;        // JVP: laid out like pix (fp32); NULL selects the VJP
    float* dtheta;               // JVP: count x 5
    uint32_t* status;            // count, or NULL
    unsigned int* queue;         // work counter (zeroed before launch)
    VjpCoef* coef;               // VJP: count per-stamp coefficients (scratch)
    R50Grad* r50g;               // FSE_MOM_SIGW_R50: count growth-curve records (scratch)
};

// Arguments of the cut-out launches (fse_cutout, Sec. 4.1).
struct CutoutArgs {
    const void* images;
    int dtype;
    const float* scale;          // bf16: per-image scale for the growth curve
    const fse_stamp* img_idx;
    int64_t count;
    double side_factor;
    int min_side, max_side;
    fse_cutout_info* info;
    fse_stamp* out_idx;
    void* out_pix;               // NULL: sizes and offsets only
    int64_t out_capacity;        // elements
    int64_t* out_total;          // device: elements of all cut-outs
};

// Number of nodes of the b(n) table and its range.
constexpr double kBnLo = 0.125;
constexpr double kBnStep = 1.0 / 512.0;
constexpr int kBnNodes = 5200;   // covers [0.125, 10.28]

// Device address of the fp32 b(n), b'(n) table of the current device.
const float2* bn_table_f32();
// Builds the b(n), b'(n) table of the current device (idempotent per device).
cudaError_t build_bn_table(cudaStream_t stream);
// Evaluates the table at count points (device arrays).
cudaError_t eval_bn(const double* n, double* b, double* db, int64_t count, cudaStream_t stream);
// Launches the estimator kernel; returns the launch error.
cudaError_t launch_estimator(const LaunchArgs& a, cudaStream_t stream);
// Launches the implicit-gradient kernel; returns the launch error.
cudaError_t launch_moment_grad(const MomentGradArgs& a, cudaStream_t stream);
// Launches the three cut-out kernels; returns the launch error.
cudaError_t launch_cutout(const CutoutArgs& a, cudaStream_t stream);
// Launches the star-profile kernel; returns the launch error.
cudaError_t launch_star(const StarArgs& a, cudaStream_t stream);
// Launches the chi^2 / adjoint kernel; returns the launch error.
cudaError_t launch_chi2_grad(const GradArgs& a, cudaStream_t stream);
// Shared memory of one stamp group (warps_per_stamp warps) for stamps of up
// to max_pix pixels, with the per-pixel inverse-variance tile when ivar is set.
size_t smem_per_group(int max_pix, bool ivar, int warps_per_stamp);
// Identity of the calling thread's current CUDA context (the driver's context
// id), or 0 when it cannot be had.  State kept per device for the life of the
// process (the b(n) table, the shared-memory opt-in of a kernel, the static
// scratch address) belongs to a context: after cudaDeviceReset the device's
// primary context is a new one and that state must be set up again.
unsigned long long current_context_id();
// Library launch shape for a tile size: warps per stamp, and warps per CTA
// (a multiple of it) as large as shared memory allows, up to four groups.
void choose_launch(int max_pix, int* warps_per_cta, int* warps_per_stamp);

}  // namespace fse
