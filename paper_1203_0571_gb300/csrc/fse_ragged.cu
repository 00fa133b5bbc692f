// fse_ragged.cu -- bucketing of a ragged batch into size classes on the
// device, so that each class runs in its own persistent launch with a
// shared-memory tile sized for that class (a tile sized for the largest stamp
// of the batch would leave one warp per SM for every stamp).  Counting and
// scattering aggregate per block in shared memory: one global atomic per class
// and block, not per stamp.  The order of stamps inside a class is not fixed;
// results do not depend on it (each stamp is measured on its own).
#include <cuda_runtime.h>

#include <stdint.h>

#include "fse_internal.h"

namespace fse {
namespace {

__device__ __forceinline__ int class_of(const fse_stamp& s) {
    const long long np = static_cast<long long>(s.h) * s.w;
    if (s.h < 1 || s.w < 1 || np > FSE_MAX_PIX) return 0;   // flagged without reading pixels
    static_assert(kClasses == 7, "class bounds below");
    return np <= 16 * 16 ? 0 : np <= 24 * 24 ? 1 : np <= 32 * 32 ? 2 : np <= 48 * 48 ? 3
         : np <= 64 * 64 ? 4 : np <= 96 * 96 ? 5 : 6;
}

__global__ void count_kernel(const fse_stamp* idx, int64_t count, unsigned int* counts) {
    __shared__ unsigned int c[kClasses];
    if (threadIdx.x < kClasses) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&c[class_of(idx[i])], 1u);
    __syncthreads();
    if (threadIdx.x < kClasses && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

// range[k] = {first slot of class k in perm, its count}; cursor[k] = first slot.
__global__ void scan_kernel(const unsigned int* counts, unsigned int* range, unsigned int* cursor) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned int off = 0;
    for (int k = 0; k < kClasses; ++k) {
        range[2 * k] = off;
        range[2 * k + 1] = counts[k];
        cursor[k] = off;
        off += counts[k];
    }
}

// One pass over a block-sized chunk: ranks inside the block from shared
// atomics, one reservation per class and block, then the writes.
__global__ void scatter_kernel(const fse_stamp* idx, int64_t count, unsigned int* cursor,
                               int32_t* perm) {
    __shared__ unsigned int c[kClasses];
    __shared__ unsigned int start[kClasses];
    for (int64_t b0 = blockIdx.x * static_cast<int64_t>(blockDim.x); b0 < count;
         b0 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (threadIdx.x < kClasses) c[threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = b0 + threadIdx.x;
        int k = 0;
        unsigned int rank = 0;
        if (i < count) {
            k = class_of(idx[i]);
            rank = atomicAdd(&c[k], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kClasses && c[threadIdx.x])
            start[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], c[threadIdx.x]);
        __syncthreads();
        if (i < count) perm[start[k] + rank] = static_cast<int32_t>(i);
        __syncthreads();
    }
}

}  // namespace

cudaError_t classify_stamps(const fse_stamp* idx, int64_t count, unsigned int* counts,
                            unsigned int* range, unsigned int* cursor, int32_t* perm,
                            cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256;
    long long blocks = (count + threads - 1) / threads;
    const long long cap = 8LL * (sms > 0 ? sms : 1);
    if (blocks > cap) blocks = cap;
    count_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(idx, count, counts);
    scan_kernel<<<1, 32, 0, stream>>>(counts, range, cursor);
    scatter_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(idx, count, cursor, perm);
    return cudaGetLastError();
}

}  // namespace fse
