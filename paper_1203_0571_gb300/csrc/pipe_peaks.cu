// pipe_peaks.cu -- throughput of the instruction pipes the estimator uses
// (fp32 FFMA, MUFU ex2 and lg2, fp64 DFMA with all 32 lanes or a single lane
// active), measured with register-only dependency chains.  A measurement
// helper for the roofline denominators; it computes nothing of the method.
#include <cuda_runtime.h>

#include <stdint.h>

#include "fse_peaks.h"

namespace {

constexpr int kChains = 8;

__global__ void k_ffma(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3f * (threadIdx.x + c);
    const float m = 0.999999f, k = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = -1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            a[c] = -y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_lg2(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 2.f + 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float y;
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[c]));
            a[c] = y + 2.f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// lanes: number of active lanes per warp (1 or 32)
__global__ void k_dfma(float* out, int iters, int lanes) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1e-3 * (threadIdx.x + c);
    if ((threadIdx.x & 31) < lanes) {
        const double m = 0.999999, k = 1e-7;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, k);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = static_cast<float>(s);
}

}  // namespace

extern "C" int fse_pipe_peaks(double* gops, int device) {
    if (!gops) return 1;
    if (cudaSetDevice(device) != cudaSuccess) return 2;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = sms * 8;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * threads * blocks) != cudaSuccess) return 3;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto timeit = [&](auto launch) {
        launch();
        cudaDeviceSynchronize();
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return static_cast<double>(ms) * 1e-3;
    };
    const double lanes_total = static_cast<double>(threads) * blocks;
    const int it32 = 4096, it64 = 64;
    double t = timeit([&] { k_ffma<<<blocks, threads>>>(out, it32); });
    gops[0] = lanes_total * it32 * kChains / t / 1e9;                 // fp32 FFMA lane-ops/s
    t = timeit([&] { k_ex2<<<blocks, threads>>>(out, it32 / 4); });
    gops[1] = lanes_total * (it32 / 4) * kChains / t / 1e9;           // ex2 lane-ops/s
    t = timeit([&] { k_lg2<<<blocks, threads>>>(out, it32 / 4); });
    gops[2] = lanes_total * (it32 / 4) * kChains / t / 1e9;           // lg2 lane-ops/s
    t = timeit([&] { k_dfma<<<blocks, threads>>>(out, it64, 32); });
    gops[3] = lanes_total * it64 * kChains / t / 1e9;                 // DFMA lane-ops/s, full warps
    t = timeit([&] { k_dfma<<<blocks, threads>>>(out, it64, 1); });
    gops[4] = (lanes_total / 32) * it64 * kChains / t / 1e9;          // DFMA warp-instructions/s, 1 lane
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
    gops[5] = sms;
    gops[6] = clk / 1e3;                                              // MHz (nominal max)
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
