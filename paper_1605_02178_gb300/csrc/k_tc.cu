// Fused tensor-core form of the fast algorithm.
//
//   k_build_hpass_tc : f -> channels e*u^n (eq. (6), centring eq. (17)) generated in shared
//                      memory as BF16/FP16, then the row pass of eq. (7) as a banded
//                      Toeplitz product on the tensor cores; writes the row-filtered
//                      channels Y[c][p][x] (p = padded row, image row p - P, mirrored).
//   k_vpass_combine_tc : per channel (highest first) the column pass of eq. (7) as a banded
//                      Toeplitz product with Y tiles fed by TMA through an mbarrier ring,
//                      then Horner accumulation of P and Q (eqs. (8)-(9)) in registers and
//                      the guarded ratio (eq. (10)) with un-centring.
//
// Banded Toeplitz product.  With k-blocks of 16 input samples and output blocks of 16,
// output block j only meets k-blocks j-a .. j+a (a = ceil(R/16)); the 16x16 (or 16x8)
// Toeplitz fragments depend only on the offset o = kb - j, so the (2a+1) fragments of the
// spatial kernel stay in registers for the whole kernel.  Work per output and channel:
// 16 (2a+1) multiply-adds against the 2R+1 of the direct sum (80 vs 61 at R = 30).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <type_traits>

#include "bfgc_common.cuh"
#include "bfgc_tc.h"

namespace bfgc {

// ----------------------------------------------------------------------------- helpers
template <typename T> struct Pack;
template <> struct Pack<__nv_bfloat16> {
    static __device__ __forceinline__ uint32_t two(float lo, float hi) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
};
template <> struct Pack<__half> {
    static __device__ __forceinline__ uint32_t two(float lo, float hi) {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&v);
    }
};

template <typename T>
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1);
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__half>(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t* r, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t* r, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

// spatial tap at signed offset d (zero outside the window)
__device__ __forceinline__ float tap(const Taps& t, int d) {
    const int ad = d < 0 ? -d : d;
    return ad <= t.R ? t.g[ad] : 0.0f;
}

// ----------------------------------------------------------------------------- kernel A
// Tile: TR padded rows x 256 output columns.  Shared memory holds the channels of the
// TR rows over the columns x0 - 16a .. x0 + 256 + 16a as an M x K matrix, M = TR*C rows
// (row m = r*C + c), K = 256 + 32a columns, row pitch padded by 16 bytes so that the 8
// row addresses of an ldmatrix fall in distinct bank groups.
constexpr int KA_COLS = 256;

__host__ __device__ inline int ka_kcols(int a) { return KA_COLS + 32 * a; }
__host__ __device__ inline int ka_pitch_bytes(int a) { return ka_kcols(a) * 2 + 16; }

template <typename T, int A>
__global__ void __launch_bounds__(256) k_build_hpass_tc(const float* __restrict__ f, T* __restrict__ Y,
                                                        const GcParams p, const Taps t, TcGeom g) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int TR = g.ka_rows, C = p.C;
    const int M = TR * C, MP = (M + 15) & ~15;
    const int KC = ka_kcols(A), PB = ka_pitch_bytes(A);
    const int p0 = blockIdx.y * TR;                 // first padded row of the tile
    const int x0 = blockIdx.x * KA_COLS;

    // ---- channels into shared memory: two columns per thread-iteration
    const int pairs = KC / 2;
    for (int idx = tid; idx < TR * pairs; idx += blockDim.x) {
        const int r = idx / pairs, kp = idx - r * pairs;
        const int pr = p0 + r;
        unsigned char* row = smem + (size_t)(r * C) * PB + kp * 4;
        if (pr >= g.Hp) {
            for (int c = 0; c < C; ++c) *reinterpret_cast<uint32_t*>(row + (size_t)c * PB) = 0u;
            continue;
        }
        int y = pr - g.P;
        y = (unsigned)y < (unsigned)p.H ? y : mirror(y, p.H);
        const float* frow = f + (size_t)y * p.W;
        int xa = x0 - 16 * A + 2 * kp, xb = xa + 1;
        xa = (unsigned)xa < (unsigned)p.W ? xa : mirror(xa, p.W);
        xb = (unsigned)xb < (unsigned)p.W ? xb : mirror(xb, p.W);
        const float ua = (__ldg(frow + xa) - p.t_c) * p.inv_sr, ub = (__ldg(frow + xb) - p.t_c) * p.inv_sr;
        float va = expf(-p.half_mu * ua * ua), vb = expf(-p.half_mu * ub * ub);
        for (int c = 0; c < C; ++c) {
            *reinterpret_cast<uint32_t*>(row + (size_t)c * PB) = Pack<T>::two(va, vb);
            va *= ua;
            vb *= ub;
        }
    }
    for (int idx = tid; idx < (MP - M) * (PB / 4); idx += blockDim.x) {
        const int r = M + idx / (PB / 4), w = idx % (PB / 4);
        reinterpret_cast<uint32_t*>(smem + (size_t)r * PB)[w] = 0u;
    }

    // ---- Toeplitz B fragments: B[k][n] = g(16(o - a) + k - 8h - n), o = 0..2a, h = 0, 1
    uint32_t bf[2 * A + 1][2][2];
    {
        const int gn = lane >> 2, tk = (lane & 3) * 2;
#pragma unroll
        for (int o = 0; o <= 2 * A; ++o)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int base = 16 * (o - A) - 8 * h - gn;
                bf[o][h][0] = Pack<T>::two(tap(t, base + tk), tap(t, base + tk + 1));
                bf[o][h][1] = Pack<T>::two(tap(t, base + tk + 8), tap(t, base + tk + 9));
            }
    }
    __syncthreads();

    // ---- MMA: items = (16-row M block, 64-column output group)
    const int mblocks = MP / 16, items = mblocks * 4;
    const uint32_t sbase = smem_u32(smem);
    for (int it = warp; it < items; it += 8) {
        const int mb = it >> 2, ng = it & 3;
        float acc[4][2][4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[jj][h][e] = 0.0f;
        const uint32_t arow = sbase + (uint32_t)((mb * 16 + (lane & 15)) * PB) + (uint32_t)((lane >> 4) * 16);
#pragma unroll
        for (int i = 0; i < 4 + 2 * A; ++i) {
            const int kb = 4 * ng + i;                        // local k-block
            uint32_t af[4];
            ldmatrix_x4(af, arow + (uint32_t)(kb * 32));
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int o = i - jj;
                if (o >= 0 && o <= 2 * A) {
                    mma16816<T>(acc[jj][0], af, bf[o][0][0], bf[o][0][1]);
                    mma16816<T>(acc[jj][1], af, bf[o][1][0], bf[o][1][1]);
                }
            }
        }
        // ---- epilogue: D rows -> (padded row, channel), columns -> output columns
        const int gr = lane >> 2, tc2 = (lane & 3) * 2;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int m = mb * 16 + gr + 8 * half;
            if (m >= M) continue;
            const int r = m / C, c = m - r * C;
            const int pr = p0 + r;
            if (pr >= g.Hp) continue;
            T* yrow = Y + ((size_t)c * g.Hp + pr) * g.Wp;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int x = x0 + 64 * ng + 16 * jj + 8 * h + tc2;
                    if (x < g.Wp)
                        *reinterpret_cast<uint32_t*>(yrow + x) =
                            Pack<T>::two(acc[jj][h][2 * half], acc[jj][h][2 * half + 1]);
                }
        }
    }
}

// ----------------------------------------------------------------------------- kernel B
constexpr int KB_ROWS = 64, KB_COLS = 64;
constexpr unsigned kSpinLimit = 1u << 21;      // bounded mbarrier waits (polls)

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`; false if the bounded spin ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    for (unsigned i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared layout: S stages of (64 + 32a) rows x 128 bytes (TMA 128-byte swizzle: the
// 16-byte chunk j of row r sits at chunk j ^ (r & 7)), each 1024-byte aligned, then S
// mbarriers.
__host__ __device__ inline int kb_tile_rows(int a) { return KB_ROWS + 32 * a; }
__host__ __device__ inline int kb_stage_bytes(int a) { return kb_tile_rows(a) * 128; }

template <typename T, int A>
__global__ void __launch_bounds__(256) k_vpass_combine_tc(const __grid_constant__ CUtensorMap ymap,
                                                          const float* __restrict__ f, float* __restrict__ out,
                                                          const GcParams p, const Taps t, TcGeom g,
                                                          DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128-byte swizzle pattern repeats every 1024 bytes: align the stages to it
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = g.kb_stages, C = p.C;
    const int ROWS = kb_tile_rows(A), SB = kb_stage_bytes(A);
    const int box_rows = g.kb_box_rows, loads = ROWS / box_rows;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
    const int x0 = blockIdx.x * KB_COLS, y0 = blockIdx.y * KB_ROWS;

    // channel m of the tile lives at Y rows m*Hp + y0 .. + ROWS (padded rows start P above)
    auto issue = [&](int m, int s) {
        mbar_expect_tx(&bars[s], (unsigned)SB);
        for (int l = 0; l < loads; ++l)
            tma_load_2d(smem + (size_t)s * SB + (size_t)l * box_rows * 128, &ymap, x0,
                        m * g.Hp + y0 + l * box_rows, &bars[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        for (int s = 0; s < S && s < C; ++s) issue(C - 1 - s, s);
    }

    // ---- Toeplitz A fragments: A[m][k] = g(16(o - a) + k - m), o = 0..2a
    uint32_t af[2 * A + 1][4];
    {
        const int gm = lane >> 2, tk = (lane & 3) * 2;
#pragma unroll
        for (int o = 0; o <= 2 * A; ++o) {
            const int base = 16 * (o - A) + tk - gm;
            af[o][0] = Pack<T>::two(tap(t, base), tap(t, base + 1));
            af[o][1] = Pack<T>::two(tap(t, base - 8), tap(t, base - 7));
            af[o][2] = Pack<T>::two(tap(t, base + 8), tap(t, base + 9));
            af[o][3] = Pack<T>::two(tap(t, base), tap(t, base + 1));
        }
    }

    // ---- per-thread pixels: warp (rh, cq) owns rows 32rh.. +32, columns 16cq.. +16
    const int rh = warp & 1, cq = warp >> 1;
    const int gr = lane >> 2, tc2 = (lane & 3) * 2;
    RatioAcc px[2][2][4];                          // [m16 block][n8 half][fragment element]
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int y = y0 + 32 * rh + 16 * mb + gr + 8 * (e >> 1);
                const int x = x0 + 16 * cq + 8 * h + tc2 + (e & 1);
                const float fv = (y < p.H && x < p.W) ? __ldg(f + (size_t)y * p.W + x) : p.t_c;
                px[mb][h][e].init((fv - p.t_c) * p.inv_sr);
            }
    __syncthreads();                                // barrier init visible to all threads

    bool ok = true;
    int i_fail = C;
    for (int i = 0; i < C; ++i) {
        const int m = C - 1 - i, s = i % S;
        const unsigned parity = (unsigned)((i / S) & 1);
        if (ok && !mbar_wait(&bars[s], parity)) {
            ok = false;
            i_fail = i;
            atomicOr(&diag->error_flags, 1u);
        }
        if (ok) {
            float acc[2][2][4];
#pragma unroll
            for (int mb = 0; mb < 2; ++mb)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[mb][h][e] = 0.0f;
            const unsigned char* st = smem + (size_t)s * SB;
            const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lchunk = 2 * cq + (lane >> 4);
#pragma unroll
            for (int kk = 0; kk < 2 + 2 * A; ++kk) {
                const int kb = 2 * rh + kk;
                const int row = 16 * kb + lrow;
                uint32_t b[4];
                ldmatrix_x4_trans(b, smem_u32(st + row * 128 + ((lchunk ^ (row & 7)) << 4)));
#pragma unroll
                for (int mb = 0; mb < 2; ++mb) {
                    const int o = kk - mb;
                    if (o >= 0 && o <= 2 * A) {
                        mma16816<T>(acc[mb][0], af[o], b[0], b[1]);
                        mma16816<T>(acc[mb][1], af[o], b[2], b[3]);
                    }
                }
            }
#pragma unroll
            for (int mb = 0; mb < 2; ++mb)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int e = 0; e < 4; ++e) px[mb][h][e].step(p, m, acc[mb][h][e]);
        }
        __syncthreads();                            // stage s fully consumed
        if (tid == 0 && ok && i + S < C) issue(m - S, s);
    }
    if (!ok) {
        // a load did not land in time: wait (bounded again) for the loads still in flight
        for (int j = i_fail; j < C && j < i_fail + S; ++j) mbar_wait(&bars[j % S], (unsigned)((j / S) & 1));
    }

    // ---- ratio and store
    unsigned guarded = 0, f64 = 0;
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int y = y0 + 32 * rh + 16 * mb + gr + 8 * (e >> 1);
                const int x = x0 + 16 * cq + 8 * h + tc2 + (e & 1);
                if (y < p.H && x < p.W) {
                    const float fv = __ldg(f + (size_t)y * p.W + x);
                    int how;
                    const float o = px[mb][h][e].finish(p, fv, &how);
                    out[(size_t)y * p.W + x] = ok ? o : __int_as_float(0x7fc00000);
                    guarded += how == 2;
                    f64 += how == 1;
                }
            }
    count_diag(diag, guarded, f64);
}

// ----------------------------------------------------------------------------- host side
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

template <typename T, int A>
cudaError_t launch_tc_impl(const float* f, void* Yv, float* out, const GcParams& p, const Taps& t,
                           const TcGeom& g, DiagHeader* diag, cudaStream_t s, int which) {
    T* Y = static_cast<T*>(Yv);
    if (which == 0) {
        const size_t smem = (size_t)((g.ka_rows * p.C + 15) & ~15) * ka_pitch_bytes(A);
        auto kern = k_build_hpass_tc<T, A>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((g.Wp + KA_COLS - 1) / KA_COLS, (g.Hp + g.ka_rows - 1) / g.ka_rows);
        kern<<<grid, 256, smem, s>>>(f, Y, p, t, g);
        return cudaGetLastError();
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    alignas(64) CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)g.Wp, (cuuint64_t)p.C * g.Hp};
    const cuuint64_t strides[1] = {(cuuint64_t)g.Wp * sizeof(T)};
    const cuuint32_t box[2] = {(cuuint32_t)KB_COLS, (cuuint32_t)g.kb_box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, sizeof(T) == 2 && std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     2, Yv, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = (size_t)g.kb_stages * kb_stage_bytes(A) + 64 * 8 + 1024;
    auto kern = k_vpass_combine_tc<T, A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.Wp + KB_COLS - 1) / KB_COLS, (g.Hp - 2 * g.P) / KB_ROWS);
    kern<<<grid, 256, smem, s>>>(map, f, out, p, t, g, diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tc_a(const float* f, void* Y, float* out, const GcParams& p, const Taps& t, const TcGeom& g,
                        DiagHeader* diag, cudaStream_t s, int which) {
    switch (g.a) {
    case 1: return launch_tc_impl<T, 1>(f, Y, out, p, t, g, diag, s, which);
    case 2: return launch_tc_impl<T, 2>(f, Y, out, p, t, g, diag, s, which);
    case 3: return launch_tc_impl<T, 3>(f, Y, out, p, t, g, diag, s, which);
    case 4: return launch_tc_impl<T, 4>(f, Y, out, p, t, g, diag, s, which);
    case 5: return launch_tc_impl<T, 5>(f, Y, out, p, t, g, diag, s, which);
    case 6: return launch_tc_impl<T, 6>(f, Y, out, p, t, g, diag, s, which);
    case 7: return launch_tc_impl<T, 7>(f, Y, out, p, t, g, diag, s, which);
    case 8: return launch_tc_impl<T, 8>(f, Y, out, p, t, g, diag, s, which);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

TcGeom tc_geometry(int H, int W, int R, int C) {
    TcGeom g{};
    g.a = (R + 15) / 16;
    if (g.a < 1) g.a = 1;
    g.P = 16 * g.a;
    g.Hp = (H + KB_ROWS - 1) / KB_ROWS * KB_ROWS + 2 * g.P;
    g.Wp = (W + KB_COLS - 1) / KB_COLS * KB_COLS;
    // kernel A: padded rows per tile, as many as fit ~100 KB of channel rows (at most 4)
    const int pitch = ka_pitch_bytes(g.a);
    g.ka_rows = 4;
    while (g.ka_rows > 1 && (size_t)((g.ka_rows * C + 15) & ~15) * pitch > 100 * 1024) --g.ka_rows;
    // kernel B: TMA box of at most 256 rows; stages that fit ~150 KB
    const int rows = kb_tile_rows(g.a);
    g.kb_box_rows = rows <= 256 ? rows : rows / 2;
    g.kb_stages = 4;
    while (g.kb_stages > 2 && (size_t)g.kb_stages * kb_stage_bytes(g.a) > 150 * 1024) --g.kb_stages;
    return g;
}

size_t tc_workspace_bytes(const TcGeom& g, int C) { return (size_t)C * g.Hp * g.Wp * 2; }

bool tc_supported(int R, int C) {
    if (R > 16 * BF_TC_MAX_A) return false;
    const TcGeom g = tc_geometry(64, 64, R, C);
    return (size_t)((g.ka_rows * C + 15) & ~15) * ka_pitch_bytes(g.a) <= 200 * 1024;
}

cudaError_t launch_build_hpass_tc(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                  bool fp16, cudaStream_t s) {
    return fp16 ? launch_tc_a<__half>(f, Y, nullptr, p, t, g, nullptr, s, 0)
                : launch_tc_a<__nv_bfloat16>(f, Y, nullptr, p, t, g, nullptr, s, 0);
}

cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s) {
    return fp16 ? launch_tc_a<__half>(f, Y, out, p, t, g, diag, s, 1)
                : launch_tc_a<__nv_bfloat16>(f, Y, out, p, t, g, diag, s, 1);
}

}  // namespace bfgc
