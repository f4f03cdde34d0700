// Plain (unfused) form of the fast algorithm, FP32 throughout:
//   build   : f -> channels e*u^n, n = 0..N+1          (eq. (6) after centring, eq. (17))
//   hpass   : channels -> row-filtered channels          (eq. (7), x axis, mirror extension)
//   vpass   : row-filtered -> fully filtered channels    (eq. (7), y axis, mirror extension)
//   combine : P, Q and the ratio                          (eqs. (8)-(10), un-centring)
// Channel planes are stored one after another with a stride of cs floats.
#include "bfgc_common.cuh"

namespace bfgc {

size_t plain_plane_stride(int H, int W) { return ((size_t)H * W + 63) / 64 * 64; }

// ---------------------------------------------------------------------------------------
// build: four pixels per thread, one float4 store per channel.
__global__ void __launch_bounds__(256) k_build(const float* __restrict__ f, float* __restrict__ X,
                                               const GcParams p, size_t cs, size_t px) {
    const size_t n4 = px / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const float4 v = reinterpret_cast<const float4*>(f)[q];
        const float4 u = make_float4((v.x - p.t_c) * p.inv_sr, (v.y - p.t_c) * p.inv_sr,
                                     (v.z - p.t_c) * p.inv_sr, (v.w - p.t_c) * p.inv_sr);
        float4 c = make_float4(expf(-p.half_mu * u.x * u.x), expf(-p.half_mu * u.y * u.y),
                               expf(-p.half_mu * u.z * u.z), expf(-p.half_mu * u.w * u.w));
        float4* dst = reinterpret_cast<float4*>(X) + q;
        for (int n = 0; n < p.C; ++n) {
            dst[(size_t)n * (cs / 4)] = c;
            c.x *= u.x; c.y *= u.y; c.z *= u.z; c.w *= u.w;
        }
    }
    const size_t i = n4 * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < px) {
        const float u = (f[i] - p.t_c) * p.inv_sr;
        float c = expf(-p.half_mu * u * u);
        for (int n = 0; n < p.C; ++n) {
            X[(size_t)n * cs + i] = c;
            c *= u;
        }
    }
}

cudaError_t launch_build(const float* f, float* X, const GcParams& p, size_t cs, cudaStream_t s) {
    const size_t px = (size_t)p.H * p.W;
    const size_t n4 = px / 4;
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n4 + 255) / 256, 152 * 16));
    k_build<<<blocks, 256, 0, s>>>(f, X, p, cs, px);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Row pass.  A block filters a 32-row x 256-column tile of one plane.  Lane = row,
// warp = 32-column slab; each thread produces 8 consecutive outputs at a time from a
// sliding register window (2 LDS.128 + 2 broadcast LDS.128 per 64 FMA).
constexpr int HP_ROWS = 32, HP_COLS = 256;

__host__ __device__ inline int hpass_len(int R) { return (HP_COLS + 2 * R + 8 + 3) / 4 * 4; }
__host__ __device__ inline int hpass_pitch(int R) {
    int p = hpass_len(R);
    while (p % 32 != 4) p += 4;          // LDS.128 across 8 lanes hits 8 distinct 16-B slots
    return p;
}
__host__ __device__ inline int taps_len(int R) { return (2 * R + 1 + 7) / 8 * 8; }

// Adjoint of eq. (7) along one axis (the backward pass): with symmetric taps the transpose of
// "mirror-extend, then filter" is "zero-extend, then filter" plus, for each output j within R
// of an end, the contributions that the forward sent to the mirror images of j, folded back:
//   sum over images p != j of j in [-R, n-1+R] of sum_{i in [0,n), |p-i| <= R} g(p-i) x(i),
// images p = j + 2nk and p = -1 - j + 2nk.  Reads `line` (stride `step`) from global memory;
// only outputs near the ends call it.
__device__ float fold_back(const float* __restrict__ line, size_t step, int j, int n, const Taps& t) {
    const int R = t.R, period = 2 * n;
    float acc = 0.0f;
    for (int k = -((R + n) / period) - 1; k <= (R + n) / period + 1; ++k) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            const long pp = sgn == 0 ? (long)j + (long)period * k : -1L - j + (long)period * k;
            if (pp == j || pp < -R || pp > n - 1 + R) continue;
            const int ip = (int)pp;
            const int lo = ip - R < 0 ? 0 : ip - R, hi = ip + R < n - 1 ? ip + R : n - 1;
            for (int i = lo; i <= hi; ++i) acc = fmaf(t.g[abs(ip - i)], line[(size_t)i * step], acc);
        }
    }
    return acc;
}

// ADJ = false: eq. (7) along x with mirror extension; ADJ = true: its adjoint (zero extension and
// the mirror images folded back, see fold_back).
template <bool ADJ>
__global__ void __launch_bounds__(256) k_hpass(const float* __restrict__ X, float* __restrict__ Y,
                                               const GcParams p, const Taps t, size_t cs) {
    extern __shared__ __align__(16) float smem[];
    const int R = t.R, W = p.W, H = p.H;
    const int LEN = hpass_len(R), PITCH = hpass_pitch(R), T = taps_len(R);
    float* s = smem;                              // [HP_ROWS][PITCH]
    float* g = smem + HP_ROWS * PITCH;            // [T]: g[d] = tap(d - R), zero beyond 2R
    const int x0 = blockIdx.x * HP_COLS, y0 = blockIdx.y * HP_ROWS;
    const float* src = X + (size_t)blockIdx.z * cs;
    float* dst = Y + (size_t)blockIdx.z * cs;
    const int tid = threadIdx.x;

    for (int d = tid; d < T; d += blockDim.x) g[d] = d <= 2 * R ? t.g[abs(d - R)] : 0.0f;
    {
        // warp w loads rows w, w+8, ...; lanes stride along the row (mirror only at the edges)
        const int lane = tid & 31, warp = tid >> 5;
        for (int r = warp; r < HP_ROWS; r += 8) {
            const int y = y0 + r;
            float* srow = s + r * PITCH;
            if (y < H) {
                const float* grow = src + (size_t)y * W;
                for (int k = lane; k < LEN; k += 32) {
                    const int x = x0 - R + k;
                    if (ADJ) srow[k] = (unsigned)x < (unsigned)W ? grow[x] : 0.0f;
                    else srow[k] = grow[(unsigned)x < (unsigned)W ? x : mirror(x, W)];
                }
            } else {
                for (int k = lane; k < LEN; k += 32) srow[k] = 0.0f;
            }
        }
    }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const float* srow = s + lane * PITCH;
    float4 res[8];
#pragma unroll
    for (int vb = 0; vb < 4; ++vb) {
        const int xb = warp * 32 + vb * 8;
        float acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0.0f;
        for (int d0 = 0; d0 < T; d0 += 8) {
            float w0[8], w1[8], gg[8];
            *reinterpret_cast<float4*>(&w0[0]) = *reinterpret_cast<const float4*>(srow + xb + d0);
            *reinterpret_cast<float4*>(&w0[4]) = *reinterpret_cast<const float4*>(srow + xb + 4 + d0);
            *reinterpret_cast<float4*>(&w1[0]) = *reinterpret_cast<const float4*>(srow + xb + 8 + d0);
            *reinterpret_cast<float4*>(&w1[4]) = *reinterpret_cast<const float4*>(srow + xb + 12 + d0);
            *reinterpret_cast<float4*>(&gg[0]) = *reinterpret_cast<const float4*>(g + d0);
            *reinterpret_cast<float4*>(&gg[4]) = *reinterpret_cast<const float4*>(g + d0 + 4);
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[v] = fmaf(gg[j], (v + j < 8) ? w0[v + j] : w1[v + j - 8], acc[v]);
        }
        res[2 * vb] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        res[2 * vb + 1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();                              // everyone done reading the input tile
    float* o = s;                                 // reuse as [HP_ROWS][PITCH] output staging
#pragma unroll
    for (int vb = 0; vb < 4; ++vb) {
        *reinterpret_cast<float4*>(o + lane * PITCH + warp * 32 + vb * 8) = res[2 * vb];
        *reinterpret_cast<float4*>(o + lane * PITCH + warp * 32 + vb * 8 + 4) = res[2 * vb + 1];
    }
    __syncthreads();
    for (int idx = tid; idx < HP_ROWS * HP_COLS; idx += blockDim.x) {
        const int r = idx / HP_COLS, c = idx - r * HP_COLS;
        const int y = y0 + r, x = x0 + c;
        if (y < H && x < W) {
            float v = o[r * PITCH + c];
            if (ADJ && (x < R || x > W - 1 - R)) v += fold_back(src + (size_t)y * W, 1, x, W, t);
            dst[(size_t)y * W + x] = v;
        }
    }
}

template <bool ADJ>
cudaError_t launch_hpass_t(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs, int planes,
                           cudaStream_t s) {
    const size_t smem = (size_t)(HP_ROWS * hpass_pitch(t.R) + taps_len(t.R)) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_hpass<ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + HP_COLS - 1) / HP_COLS, (p.H + HP_ROWS - 1) / HP_ROWS, planes);
    k_hpass<ADJ><<<grid, 256, smem, s>>>(X, Y, p, t, cs);
    return cudaGetLastError();
}

cudaError_t launch_hpass(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                         int planes, cudaStream_t s) {
    return launch_hpass_t<false>(X, Y, p, t, cs, planes, s);
}

cudaError_t launch_hpass_adjoint(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                 int planes, cudaStream_t s) {
    return launch_hpass_t<true>(X, Y, p, t, cs, planes, s);
}

// ---------------------------------------------------------------------------------------
// Column pass.  A block filters 64 output rows x 64 columns of one plane; thread = one
// column and 16 consecutive output rows (two blocks of 8 from a sliding window).
constexpr int VP_ROWS = 64, VP_COLS = 64;

__host__ __device__ inline int vpass_len(int R) { return VP_ROWS + 2 * R + 8; }

template <bool ADJ>
__global__ void __launch_bounds__(256) k_vpass(const float* __restrict__ X, float* __restrict__ Y,
                                               const GcParams p, const Taps t, size_t cs) {
    extern __shared__ __align__(16) float smem[];
    const int R = t.R, W = p.W, H = p.H;
    const int LEN = vpass_len(R), T = taps_len(R);
    float* s = smem;                              // [LEN][VP_COLS]
    float* g = smem + LEN * VP_COLS;
    const int x0 = blockIdx.x * VP_COLS, y0 = blockIdx.y * VP_ROWS;
    const float* src = X + (size_t)blockIdx.z * cs;
    float* dst = Y + (size_t)blockIdx.z * cs;
    const int tid = threadIdx.x;

    for (int d = tid; d < T; d += blockDim.x) g[d] = d <= 2 * R ? t.g[abs(d - R)] : 0.0f;
    {
        const int c = tid & (VP_COLS - 1), x = x0 + c;
        for (int r = tid / VP_COLS; r < LEN; r += 256 / VP_COLS) {
            const int y = y0 - R + r;
            if (ADJ) s[r * VP_COLS + c] = x < W && (unsigned)y < (unsigned)H ? src[(size_t)y * W + x] : 0.0f;
            else s[r * VP_COLS + c] = x < W ? src[(size_t)((unsigned)y < (unsigned)H ? y : mirror(y, H)) * W + x] : 0.0f;
        }
    }
    __syncthreads();

    const int c = tid & (VP_COLS - 1), rg = tid / VP_COLS;
#pragma unroll
    for (int vb = 0; vb < 2; ++vb) {
        const int rb = rg * 16 + vb * 8;
        float acc[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[v] = 0.0f;
        for (int d0 = 0; d0 < T; d0 += 8) {
            float w0[8], w1[8], gg[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                w0[v] = s[(rb + d0 + v) * VP_COLS + c];
                w1[v] = s[(rb + 8 + d0 + v) * VP_COLS + c];
            }
            *reinterpret_cast<float4*>(&gg[0]) = *reinterpret_cast<const float4*>(g + d0);
            *reinterpret_cast<float4*>(&gg[4]) = *reinterpret_cast<const float4*>(g + d0 + 4);
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[v] = fmaf(gg[j], (v + j < 8) ? w0[v + j] : w1[v + j - 8], acc[v]);
        }
        const int x = x0 + c;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int y = y0 + rb + v;
            if (y < H && x < W) {
                if (ADJ && (y < R || y > H - 1 - R)) acc[v] += fold_back(src + x, (size_t)W, y, H, t);
                dst[(size_t)y * W + x] = acc[v];
            }
        }
    }
}

template <bool ADJ>
cudaError_t launch_vpass_t(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs, int planes,
                           cudaStream_t s) {
    const size_t smem = (size_t)(vpass_len(t.R) * VP_COLS + taps_len(t.R)) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_vpass<ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + VP_COLS - 1) / VP_COLS, (p.H + VP_ROWS - 1) / VP_ROWS, planes);
    k_vpass<ADJ><<<grid, 256, smem, s>>>(X, Y, p, t, cs);
    return cudaGetLastError();
}

cudaError_t launch_vpass(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                         int planes, cudaStream_t s) {
    return launch_vpass_t<false>(X, Y, p, t, cs, planes, s);
}

cudaError_t launch_vpass_adjoint(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                 int planes, cudaStream_t s) {
    return launch_vpass_t<true>(X, Y, p, t, cs, planes, s);
}

// ---------------------------------------------------------------------------------------
// Ratio: Horner in u over the channels (highest first), P and Q of eqs. (8)-(9) with the
// rescaled coefficients, the division of eq. (10) (guarded, or the pixel listed for the FP64
// refinement; see GcParams), un-centring.
__global__ void __launch_bounds__(256) k_combine(const float* __restrict__ f, const float* __restrict__ Z,
                                                 float* __restrict__ out, const GcParams p, size_t cs,
                                                 size_t px, DiagHeader* diag) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t n4 = (px + 3) / 4;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const size_t i0 = q * 4;
        const bool full = i0 + 4 <= px;
        float fv[4], z[4];
        if (full) {
            *reinterpret_cast<float4*>(fv) = *reinterpret_cast<const float4*>(f + i0);
        } else {
            for (int k = 0; k < 4; ++k) fv[k] = i0 + k < px ? f[i0 + k] : p.t_c;
        }
        RatioAcc acc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k].init((fv[k] - p.t_c) * p.inv_sr);
        for (int m = p.C - 1; m >= 0; --m) {
            const float* zm = Z + (size_t)m * cs + i0;
            if (full) {
                *reinterpret_cast<float4*>(z) = *reinterpret_cast<const float4*>(zm);
            } else {
                for (int k = 0; k < 4; ++k) z[k] = i0 + k < px ? zm[k] : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k].step(p, m, z[k]);
        }
        float o[4];
        int how[4];
        unsigned guarded = 0, illcond = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[k] = acc[k].finish(p, fv[k], &how[k]);
            if (i0 + k < px) {
                guarded += how[k] == 2;
                illcond += how[k] == 1;
            }
        }
        if (full) {
            *reinterpret_cast<float4*>(out + i0) = *reinterpret_cast<float4*>(o);
        } else {
            for (int k = 0; k < 4; ++k)
                if (i0 + k < px) out[i0 + k] = o[k];
        }
        count_diag(diag, guarded, illcond);
        if (p.refine) {
#pragma unroll
            for (int k = 0; k < 4; ++k) refine_push(p, diag, i0 + k < px && how[k] == 3, (uint32_t)(i0 + k));
        }
    }
}

cudaError_t launch_combine(const float* f, const float* Z, float* out, const GcParams& p, size_t cs,
                           DiagHeader* diag, cudaStream_t s) {
    const size_t px = (size_t)p.H * p.W;
    const size_t n4 = (px + 3) / 4;
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n4 + 255) / 256, 152 * 16));
    k_combine<<<blocks, 256, 0, s>>>(f, Z, out, p, cs, px, diag);
    return cudaGetLastError();
}

}  // namespace bfgc
