// Fused form on the FP32 ALUs: two kernels instead of the plain form's four, FP32 throughout.
//   build_hpass_f32   : f -> row-filtered channels e*u^n, n = 0..N+1   (eqs. (6), (17) and the
//                       x axis of eq. (7)); the channels exist only in shared memory before
//                       the row pass, which takes them two at a time (packed f32x2 FMA).
//   vpass_combine_f32 : row-filtered channels -> P, Q and the ratio      (the y axis of eq. (7),
//                       eqs. (8)-(10)); the filtered channels exist only in registers.
// Each output takes the same FP32 operations in the same order as in the plain form (channel
// n = (e * u) * u ... built by repeated products, taps summed in ascending offset from zero,
// Horner over the channels from the highest), so the two forms agree bit for bit; this form
// saves the plain form's channel build pass, one read and one write of every channel plane,
// and the separate ratio pass.
#include "bfgc_common.cuh"

namespace bfgc {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Copy of `bytes` (4 or 16) from global to shared memory; the bytes past `src_bytes` are
// zero-filled (src_bytes = 0 reads nothing).
__device__ __forceinline__ void cp_async16(float* dst, const float* src, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" :: "r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" :: "r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" :: "n"(N) : "memory");
}

__host__ __device__ inline int taps_len8(int R) { return (2 * R + 1 + 7) / 8 * 8; }

// ---------------------------------------------------------------------------------------
// Row pass geometry: a block covers FR_ROWS rows x FR_COLS output columns and two channels at a
// time.  The two channels are interleaved in shared memory, so one LDS.128 gives two aligned
// (channel n, channel n+1) pairs and one packed fma.rn.f32x2 does the multiply-add of both
// channels (each lane takes the same FP32 operation as the plain row pass).  Lane = row, warp =
// 16-column slab, each thread produces its 16 output pairs in one sweep of a 24-pair window
// (12 LDS.128 + 4 broadcast LDS.128 per 128 packed FMA).
constexpr int FR_ROWS = 32, FR_COLS = 128, FR_WARPS = FR_COLS / 16, FR_THREADS = FR_WARPS * 32;
constexpr int FR_STAGE_PITCH = 2 * FR_COLS + 4;     // staging rows of output pairs (pitch % 8 == 4)

__host__ __device__ inline int fr_len(int R) { return (FR_COLS + 2 * R + 8 + 3) / 4 * 4; }
__host__ __device__ inline int fr_pair_pitch(int R) {
    int p = 2 * fr_len(R);
    while (p % 8 != 4) p += 4;                      // LDS.128 across 8 lanes: 8 distinct 16-B slots
    return p;
}
__host__ __device__ inline int fr_u_pitch(int R) {
    int p = fr_len(R);
    while (p % 8 != 4) p += 4;
    return p;
}
size_t fr_smem(int R) {
    return ((size_t)FR_ROWS * (fr_pair_pitch(R) + fr_u_pitch(R) + FR_STAGE_PITCH) + 2 * taps_len8(R)) * sizeof(float);
}

// ---------------------------------------------------------------------------------------
// Column pass geometry: a block covers FC_ROWS output rows x 64 columns; thread = one column
// and 16 consecutive output rows (one sweep of a 24-value window, conflict-free LDS.32).
constexpr int FC_ROWS = 64, FC_COLS = 64, FC_THREADS = 256, FC_OUT = 16;

__host__ __device__ inline int fc_len(int R) { return FC_ROWS + 2 * R + 8; }
size_t fc_smem(int R) {
    return ((size_t)2 * fc_len(R) * FC_COLS + (size_t)FC_ROWS * FC_COLS + taps_len8(R)) * sizeof(float);
}

constexpr size_t kMaxSmem = 227 * 1024;

}  // namespace

bool fused_f32_supported(int R) { return R >= 0 && R <= BF_MAX_R && fr_smem(R) <= kMaxSmem && fc_smem(R) <= kMaxSmem; }

// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t f2fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__global__ void __launch_bounds__(FR_THREADS, 2)
k_build_hpass_f32(const float* __restrict__ f, float* __restrict__ Y, const GcParams p, const Taps t, size_t cs) {
    extern __shared__ __align__(16) float smem[];
    const int R = t.R, W = p.W, H = p.H, C = p.C;
    const int LEN = fr_len(R), PP = fr_pair_pitch(R), UP = fr_u_pitch(R), T = taps_len8(R);
    float* pl = smem;                                  // [FR_ROWS][PP]: (channel n, n+1) pairs over the window
    float* us = pl + FR_ROWS * PP;                     // [FR_ROWS][UP]: u over the window
    float* st = us + FR_ROWS * UP;                     // [FR_ROWS][FR_STAGE_PITCH]: output pairs
    float* g2 = st + FR_ROWS * FR_STAGE_PITCH;         // [T][2]: (tap(d - R), tap(d - R)), zero beyond 2R
    const int x0 = blockIdx.x * FR_COLS, y0 = blockIdx.y * FR_ROWS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int d = tid; d < T; d += FR_THREADS) {
        const float v = d <= 2 * R ? t.g[abs(d - R)] : 0.0f;
        *reinterpret_cast<float2*>(g2 + 2 * d) = make_float2(v, v);
    }
    // u, channel 0 and channel 1 over the window (mirror extension along x)
    for (int r = warp; r < FR_ROWS; r += FR_WARPS) {
        const int y = y0 + r;
        float* prow = pl + r * PP;
        float* urow = us + r * UP;
        if (y < H) {
            const float* frow = f + (size_t)y * W;
            for (int k = lane; k < LEN; k += 32) {
                const int x = x0 - R + k;
                const float u = (frow[(unsigned)x < (unsigned)W ? x : mirror(x, W)] - p.t_c) * p.inv_sr;
                const float e = expf(-p.half_mu * u * u);
                urow[k] = u;
                *reinterpret_cast<float2*>(prow + 2 * k) = make_float2(e, e * u);
            }
        } else {
            for (int k = lane; k < LEN; k += 32) {
                urow[k] = 0.0f;
                *reinterpret_cast<float2*>(prow + 2 * k) = make_float2(0.0f, 0.0f);
            }
        }
    }
    __syncthreads();

    const float* wrow = pl + lane * PP + 2 * (warp * 16);
    for (int n = 0; n < C; n += 2) {
        uint64_t acc[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) acc[v] = 0ull;
        for (int d0 = 0; d0 < T; d0 += 8) {
            uint64_t w[24], tp[8];
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(wrow + 2 * d0 + 4 * q);
                w[2 * q] = v.x;
                w[2 * q + 1] = v.y;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(g2 + 2 * d0 + 4 * q);
                tp[2 * q] = v.x;
                tp[2 * q + 1] = v.y;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int v = 0; v < 16; ++v) acc[v] = f2fma(tp[j], w[v + j], acc[v]);
        }
        __syncthreads();                               // every thread is done reading this pair
        float* so = st + lane * FR_STAGE_PITCH + 2 * (warp * 16);
#pragma unroll
        for (int v = 0; v < 16; v += 2)
            *reinterpret_cast<ulonglong2*>(so + 2 * v) = make_ulonglong2(acc[v], acc[v + 1]);
        if (n + 2 < C) {                               // (n+2, n+3) = (c_{n+1} u, c_{n+1} u u), in place
            for (int r = warp; r < FR_ROWS; r += FR_WARPS) {
                float* prow = pl + r * PP;
                const float* urow = us + r * UP;
                for (int k = 2 * lane; k < LEN; k += 64) {   // window positions k, k + 1
                    float4 c = *reinterpret_cast<float4*>(prow + 2 * k);
                    const float2 u = *reinterpret_cast<const float2*>(urow + k);
                    c.x = c.y * u.x; c.y = c.x * u.x;
                    c.z = c.w * u.y; c.w = c.z * u.y;
                    *reinterpret_cast<float4*>(prow + 2 * k) = c;
                }
            }
        }
        __syncthreads();
        // staged output pairs -> planes n and n+1, row-major and coalesced
        float* dst0 = Y + (size_t)n * cs;
        float* dst1 = n + 1 < C ? dst0 + cs : nullptr;
        constexpr int Q4 = FR_COLS / 4;
        for (int i = tid; i < FR_ROWS * Q4; i += FR_THREADS) {
            const int r = i / Q4, c = (i - r * Q4) * 4;
            const int y = y0 + r, x = x0 + c;
            if (y >= H || x >= W) continue;
            const float4 lo = *reinterpret_cast<const float4*>(st + r * FR_STAGE_PITCH + 2 * c);
            const float4 hi = *reinterpret_cast<const float4*>(st + r * FR_STAGE_PITCH + 2 * c + 4);
            const float4 va = make_float4(lo.x, lo.z, hi.x, hi.z), vb = make_float4(lo.y, lo.w, hi.y, hi.w);
            const size_t o = (size_t)y * W + x;
            if ((W & 3) == 0) {
                *reinterpret_cast<float4*>(dst0 + o) = va;
                if (dst1) *reinterpret_cast<float4*>(dst1 + o) = vb;
            } else {
                const float a4[4] = {va.x, va.y, va.z, va.w}, b4[4] = {vb.x, vb.y, vb.z, vb.w};
                for (int e = 0; e < 4 && x + e < W; ++e) {
                    dst0[o + e] = a4[e];
                    if (dst1) dst1[o + e] = b4[e];
                }
            }
        }
        // the next pass over `st` starts after the first barrier of the next pair, which every
        // thread reaches only after its copy above
    }
}

// ---------------------------------------------------------------------------------------
// Issue the copies of the column window of channel plane `src` (rows y0 - R .. y0 - R + LEN - 1,
// mirrored into [0, H); columns x0 .. x0 + 63, zero past W) into `dst` [LEN][64].
template <bool VEC>
__device__ __forceinline__ void fc_issue(float* dst, const float* __restrict__ src, int x0, int y0, int R, int LEN,
                                         int H, int W, int tid) {
    if (VEC) {                                          // W % 4 == 0: 16-byte rows of 16 chunks
        const int q = tid & 15, x = x0 + 4 * q;
        const unsigned bytes = x < W ? 16u : 0u;
        for (int r = tid >> 4; r < LEN; r += FC_THREADS / 16) {
            const int y = y0 - R + r;
            const float* row = src + (size_t)((unsigned)y < (unsigned)H ? y : mirror(y, H)) * W;
            cp_async16(dst + r * FC_COLS + 4 * q, bytes ? row + x : row, bytes);
        }
    } else {
        const int c = tid & 63, x = x0 + c;
        const unsigned bytes = x < W ? 4u : 0u;
        for (int r = tid >> 6; r < LEN; r += FC_THREADS / 64) {
            const int y = y0 - R + r;
            const float* row = src + (size_t)((unsigned)y < (unsigned)H ? y : mirror(y, H)) * W;
            cp_async4(dst + r * FC_COLS + c, bytes ? row + x : row, bytes);
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(FC_THREADS, 2)
k_vpass_combine_f32(const float* __restrict__ f, const float* __restrict__ Y, float* __restrict__ out,
                    const GcParams p, const Taps t, size_t cs, DiagHeader* diag) {
    extern __shared__ __align__(16) float smem[];
    const int R = t.R, W = p.W, H = p.H;
    const int LEN = fc_len(R), T = taps_len8(R);
    float* buf0 = smem;                                 // [LEN][64], channel window, two stages
    float* buf1 = buf0 + LEN * FC_COLS;
    float* us = buf1 + LEN * FC_COLS;                   // [FC_ROWS][64]: u of the output pixels
    float* g = us + FC_ROWS * FC_COLS;                  // [T]
    const int x0 = blockIdx.x * FC_COLS, y0 = blockIdx.y * FC_ROWS;
    const int tid = threadIdx.x;
    const int C = p.C;

    fc_issue<VEC>(buf0, Y + (size_t)(C - 1) * cs, x0, y0, R, LEN, H, W, tid);
    cp_async_commit();
    for (int d = tid; d < T; d += FC_THREADS) g[d] = d <= 2 * R ? t.g[abs(d - R)] : 0.0f;
    for (int i = tid; i < FC_ROWS * FC_COLS; i += FC_THREADS) {
        const int r = i / FC_COLS, c = i - r * FC_COLS;
        const int y = y0 + r, x = x0 + c;
        us[i] = y < H && x < W ? (f[(size_t)y * W + x] - p.t_c) * p.inv_sr : 0.0f;
    }

    const int c = tid & (FC_COLS - 1), rb = (tid / FC_COLS) * FC_OUT;
    float P[FC_OUT], Q[FC_OUT], Qa[FC_OUT];
#pragma unroll
    for (int v = 0; v < FC_OUT; ++v) P[v] = Q[v] = Qa[v] = 0.0f;

    for (int i = 0; i < C; ++i) {
        const int m = C - 1 - i;                        // Horner: highest channel first
        if (i + 1 < C) {
            fc_issue<VEC>((i & 1) ? buf0 : buf1, Y + (size_t)(m - 1) * cs, x0, y0, R, LEN, H, W, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();                                // window of channel m complete and visible
        const float* s = ((i & 1) ? buf1 : buf0) + rb * FC_COLS + c;
        float acc[FC_OUT];
#pragma unroll
        for (int v = 0; v < FC_OUT; ++v) acc[v] = 0.0f;
        for (int d0 = 0; d0 < T; d0 += 8) {
            float w[FC_OUT + 8], gg[8];
#pragma unroll
            for (int v = 0; v < FC_OUT + 8; ++v) w[v] = s[(d0 + v) * FC_COLS];
            *reinterpret_cast<float4*>(&gg[0]) = *reinterpret_cast<const float4*>(g + d0);
            *reinterpret_cast<float4*>(&gg[4]) = *reinterpret_cast<const float4*>(g + d0 + 4);
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int v = 0; v < FC_OUT; ++v) acc[v] = fmaf(gg[j], w[v + j], acc[v]);
        }
        // eqs. (8)-(9): the plain ratio pass's step for channel m
        const float cm1 = m >= 1 ? p.coef[m - 1] : 0.0f, cm = p.coef[m];
#pragma unroll
        for (int v = 0; v < FC_OUT; ++v) {
            const float u = us[(rb + v) * FC_COLS + c];
            if (m >= 1) P[v] = fmaf(P[v], u, cm1 * acc[v]);
            if (m <= p.N) {
                const float q = cm * acc[v];
                Q[v] = fmaf(Q[v], u, q);
                Qa[v] = fmaf(Qa[v], fabsf(u), fabsf(q));
            }
        }
        __syncthreads();                                // every thread is done with this stage
    }

    // eq. (10) with the division guard, as the plain ratio pass
    unsigned guarded = 0, illcond = 0;
    const int x = x0 + c;
#pragma unroll
    for (int v = 0; v < FC_OUT; ++v) {
        const int y = y0 + rb + v;
        if (y < H && x < W) {
            const size_t i = (size_t)y * W + x;
            RatioAcc a;
            a.u = us[(rb + v) * FC_COLS + c];
            a.au = fabsf(a.u);
            a.P = P[v];
            a.Q = Q[v];
            a.Qa = Qa[v];
            int how;
            out[i] = a.finish(p, f[i], &how);
            guarded += how == 2;
            illcond += how == 1;
            if (p.refine) refine_push(p, diag, how == 3, (uint32_t)i);
        }
    }
    count_diag(diag, guarded, illcond);
}

// ---------------------------------------------------------------------------------------
cudaError_t launch_build_hpass_f32(const float* f, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                   cudaStream_t s) {
    if (!fused_f32_supported(t.R)) return cudaErrorInvalidValue;
    const size_t smem = fr_smem(t.R);
    cudaError_t e = cudaFuncSetAttribute(k_build_hpass_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + FR_COLS - 1) / FR_COLS, (p.H + FR_ROWS - 1) / FR_ROWS);
    k_build_hpass_f32<<<grid, FR_THREADS, smem, s>>>(f, Y, p, t, cs);
    return cudaGetLastError();
}

cudaError_t launch_vpass_combine_f32(const float* f, const float* Y, float* out, const GcParams& p, const Taps& t,
                                     size_t cs, DiagHeader* diag, cudaStream_t s) {
    if (!fused_f32_supported(t.R)) return cudaErrorInvalidValue;
    const size_t smem = fc_smem(t.R);
    dim3 grid((p.W + FC_COLS - 1) / FC_COLS, (p.H + FC_ROWS - 1) / FC_ROWS);
    cudaError_t e;
    if ((p.W & 3) == 0) {
        e = cudaFuncSetAttribute(k_vpass_combine_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_vpass_combine_f32<true><<<grid, FC_THREADS, smem, s>>>(f, Y, out, p, t, cs, diag);
    } else {
        e = cudaFuncSetAttribute(k_vpass_combine_f32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_vpass_combine_f32<false><<<grid, FC_THREADS, smem, s>>>(f, Y, out, p, t, cs, diag);
    }
    return cudaGetLastError();
}

}  // namespace bfgc
