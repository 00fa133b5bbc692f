/*
 * fse_peaks.h -- pipe-throughput microbenchmark (libfse_peaks.so).
 *
 * Not part of the paper's method (the paper has no counterpart): it measures
 * the GB300 instruction pipes the estimator runs on, to give its fp32-issue
 * roofline a measured denominator.
 */
#ifndef FSE_PEAKS_H
#define FSE_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Runs register-only dependency-chain kernels on `device` (8 blocks of 256
 * threads per SM) and writes into gops[0..6] (host array of >= 7 doubles):
 *   [0] fp32 FFMA lane-ops/s / 1e9      [1] MUFU ex2 lane-ops/s / 1e9
 *   [2] MUFU lg2 lane-ops/s / 1e9       [3] fp64 DFMA lane-ops/s / 1e9 (32 lanes)
 *   [4] fp64 DFMA warp-instructions/s / 1e9 with one active lane per warp
 *   [5] SM count                        [6] maximum SM clock, MHz
 * Returns 0 on success, non-zero on a CUDA error.  Synchronises the device. */
int fse_pipe_peaks(double *gops, int device);

#ifdef __cplusplus
}
#endif

#endif /* FSE_PEAKS_H */
