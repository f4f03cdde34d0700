// The exact Gaussian bilateral filter of eq. (1) by brute force: for every pixel the
// (2R+1)^2 window with the spatial weight exp(-|j|^2 / 2 sigma_s^2) and the range weight
// exp(-(f(i-j) - f(i))^2 / 2 sigma_r^2), half-sample mirror extension, FP32.
// Both weights are combined in one exp2 per neighbour.
#include "bfgc_common.cuh"

namespace bfgc {

constexpr int DT = 32;           // output tile (DT x DT), 256 threads, 4 outputs per thread
constexpr int DIRECT_SMEM_MAX = 215 * 1024;

__host__ __device__ inline int direct_span(int R) { return DT + 2 * R; }

// Tile of the (mirrored) input plus log2 spatial weights in shared memory.
__global__ void __launch_bounds__(256) k_direct_smem(const float* __restrict__ f, float* __restrict__ out,
                                                     int H, int W, int R, float ls_scale, float lr_scale) {
    extern __shared__ float smem[];
    const int S = direct_span(R);
    float* tile = smem;                    // [S][S]
    float* ls = smem + S * S;              // ls[d + R] = -d^2 log2(e) / (2 sigma_s^2)
    const int x0 = blockIdx.x * DT, y0 = blockIdx.y * DT, tid = threadIdx.x;
    for (int d = tid; d <= 2 * R; d += blockDim.x) ls[d] = -(float)((d - R) * (d - R)) * ls_scale;
    for (int idx = tid; idx < S * S; idx += blockDim.x) {
        const int r = idx / S, c = idx - r * S;
        tile[idx] = f[(size_t)mirror(y0 - R + r, H) * W + mirror(x0 - R + c, W)];
    }
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;          // rows ty, ty+8, ty+16, ty+24
    float fi[4], num[4], den[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        fi[k] = tile[(ty + 8 * k + R) * S + tx + R];
        num[k] = 0.0f;
        den[k] = 0.0f;
    }
    for (int dy = 0; dy <= 2 * R; ++dy) {
        const float wy = ls[dy];
        for (int dx = 0; dx <= 2 * R; ++dx) {
            const float wxy = wy + ls[dx];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float t = tile[(ty + 8 * k + dy) * S + tx + dx];
                const float df = t - fi[k];
                const float w = exp2f(fmaf(-lr_scale * df, df, wxy));
                num[k] = fmaf(w, t, num[k]);
                den[k] += w;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int y = y0 + ty + 8 * k, x = x0 + tx;
        if (y < H && x < W) out[(size_t)y * W + x] = num[k] / den[k];
    }
}

// Fallback for windows too wide for shared memory: neighbours read through the cache.
__global__ void __launch_bounds__(256) k_direct_global(const float* __restrict__ f, float* __restrict__ out,
                                                       int H, int W, int R, float ls_scale, float lr_scale) {
    const int x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (x >= W || y >= H) return;
    const float fi = f[(size_t)y * W + x];
    float num = 0.0f, den = 0.0f;
    for (int jy = -R; jy <= R; ++jy) {
        const float* row = f + (size_t)mirror(y + jy, H) * W;
        const float wy = -(float)(jy * jy) * ls_scale;
        for (int jx = -R; jx <= R; ++jx) {
            const float t = __ldg(row + mirror(x + jx, W));
            const float df = t - fi;
            const float w = exp2f(fmaf(-lr_scale * df, df, wy - (float)(jx * jx) * ls_scale));
            num = fmaf(w, t, num);
            den += w;
        }
    }
    out[(size_t)y * W + x] = num / den;
}

cudaError_t launch_direct(const float* f, float* out, int H, int W, int R, double sigma_s,
                          double sigma_r, cudaStream_t s) {
    const double log2e = 1.4426950408889634;
    const float ls_scale = (float)(log2e / (2.0 * sigma_s * sigma_s));
    const float lr_scale = (float)(log2e / (2.0 * sigma_r * sigma_r));
    const int S = direct_span(R);
    const size_t smem = ((size_t)S * S + 2 * R + 1) * sizeof(float);
    if (smem <= (size_t)DIRECT_SMEM_MAX) {
        cudaError_t e = cudaFuncSetAttribute(k_direct_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((W + DT - 1) / DT, (H + DT - 1) / DT);
        k_direct_smem<<<grid, 256, smem, s>>>(f, out, H, W, R, ls_scale, lr_scale);
    } else {
        dim3 grid((W + 15) / 16, (H + 15) / 16);
        k_direct_global<<<grid, 256, 0, s>>>(f, out, H, W, R, ls_scale, lr_scale);
    }
    return cudaGetLastError();
}

}  // namespace bfgc
