// Input range check (a diagnostic, not part of the filter): the Gauss-Chebyshev fit of the
// range kernel covers intensities in [L, U] only (Sec. III-B: the approximation interval is the
// centred dynamic range), so pixels outside it, or not finite, are outside what the filter
// approximates.  The kernel counts them and reports; it changes nothing and never traps.
#include <cuda_runtime.h>

#include "bfgc_internal.h"

namespace bfgc {

namespace {

constexpr int kChkThreads = 256;

__device__ __forceinline__ void check_one(float v, float L, float U, unsigned& outside, unsigned& nonfinite) {
    const bool fin = isfinite(v);
    nonfinite += !fin;
    outside += fin && (v < L || v > U);
}

// counts[0] += pixels outside [L, U], counts[1] += non-finite pixels
__global__ void __launch_bounds__(kChkThreads) k_check_range(const float* __restrict__ f, size_t n, float L, float U,
                                                             unsigned long long* counts) {
    unsigned outside = 0, nonfinite = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((reinterpret_cast<uintptr_t>(f) & 15) == 0) {
        const size_t n4 = n / 4;
        for (size_t k = i; k < n4; k += stride) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(f) + k);
            check_one(v.x, L, U, outside, nonfinite);
            check_one(v.y, L, U, outside, nonfinite);
            check_one(v.z, L, U, outside, nonfinite);
            check_one(v.w, L, U, outside, nonfinite);
        }
        for (size_t k = 4 * n4 + i; k < n; k += stride) check_one(__ldg(f + k), L, U, outside, nonfinite);
    } else {
        for (size_t k = i; k < n; k += stride) check_one(__ldg(f + k), L, U, outside, nonfinite);
    }
    const unsigned o = __reduce_add_sync(0xffffffffu, outside), q = __reduce_add_sync(0xffffffffu, nonfinite);
    if ((threadIdx.x & 31) == 0) {
        if (o) atomicAdd(&counts[0], (unsigned long long)o);
        if (q) atomicAdd(&counts[1], (unsigned long long)q);
    }
}

}  // namespace

cudaError_t launch_check_range(const float* f, size_t n, float L, float U, unsigned long long* counts,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n / 4 + kChkThreads - 1) / kChkThreads;
    const unsigned grid = (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)std::max(1, sms) * 8));
    k_check_range<<<grid, kChkThreads, 0, s>>>(f, n, L, U, counts);
    return cudaGetLastError();
}

}  // namespace bfgc
