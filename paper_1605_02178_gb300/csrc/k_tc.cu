// Column pass of eq. (7) + ratio (eqs. (8)-(10)) of the fused tensor-core form.
//
//   k_vpass_combine_tc : per channel (highest first) the column pass as a banded Toeplitz
//                        product on mma.sync tiles, the row-filtered channel tile fed by TMA
//                        through an mbarrier ring filled by a producer warp; Horner
//                        accumulation of P and Q in registers, then the guarded ratio and
//                        un-centring.  (The row pass is k_umma.cu.)
//
// Banded Toeplitz product.  With k-blocks of 16 input rows and output blocks of 16 rows,
// output block j only meets k-blocks j-a .. j+a (a = ceil(R/16)); the 16x16 Toeplitz
// fragments depend only on the offset o = kb - j, so the (2a+1) fragments of the spatial
// kernel stay in registers.  Work per output and channel: 16 (2a+1) multiply-adds against
// the 2R+1 of the direct sum (80 vs 61 at R = 30).
//
// Row-filtered channels Y are stored row-interleaved, Y[p][c][x] (padded row p, channel c,
// column x): the row pass writes consecutive (row, channel) product rows to consecutive
// memory rows, and the column pass reads one channel's rows with a 3-D TMA box.
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

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t* r, uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

// 13 warps (at most 4 per SM sub-partition, so 128 registers per thread are available):
// warps 0..11 compute 32x16 pixels each of a 96x64 tile, warp 12 loads.
constexpr int KB_ROWS = 96, KB_COLS = 64;
constexpr int KB_CONSUMERS = 12;
constexpr unsigned kSpinLimit = 1u << 21;          // bounded mbarrier waits (polls)

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(smem_u32(bar)) : "memory");
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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int c, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared layout: S stages of (64 + 32a) rows x 128 bytes (TMA 128-byte swizzle: the 16-byte
// chunk j of row r sits at chunk j ^ (r & 7)), each 1024-byte aligned; 2S mbarriers (full,
// empty); the taps.
__host__ __device__ inline int kb_tile_rows(int a) { return KB_ROWS + 32 * a; }
__host__ __device__ inline int kb_stage_bytes(int a) { return kb_tile_rows(a) * 128; }

template <typename T, int A>
__global__ void __launch_bounds__(32 * (KB_CONSUMERS + 1), 1) k_vpass_combine_tc(
    const __grid_constant__ CUtensorMap ymap, const float* __restrict__ f, float* __restrict__ out, const GcParams p,
    const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128-byte swizzle pattern repeats every 1024 bytes: align the stages to it
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = g.kb_stages, C = p.C;
    const int ROWS = kb_tile_rows(A), SB = kb_stage_bytes(A);
    const int box_rows = g.kb_box_rows, loads = ROWS / box_rows;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB);
    uint64_t* empty = full + S;
    float* gs = reinterpret_cast<float*>(empty + S);       // taps g[|d|], d = 0 .. 16(a+1)
    const int x0 = blockIdx.x * KB_COLS, y0 = blockIdx.y * KB_ROWS;

    for (int d = tid; d <= 16 * (A + 1); d += blockDim.x) gs[d] = d <= t.R ? t.g[d] : 0.0f;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], KB_CONSUMERS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    // ---------------------------------------------------------------- producer warp
    if (warp == KB_CONSUMERS) {
        if (lane == 0) {
            bool ok = true;
            int issued = 0;
            for (int i = 0; i < C && ok; ++i) {
                const int s = i % S, m = C - 1 - i;
                if (i >= S && !mbar_wait(&empty[s], (unsigned)(((i / S) - 1) & 1))) {
                    ok = false;
                    atomicOr(&diag->error_flags, 1u);
                    break;
                }
                mbar_expect_tx(&full[s], (unsigned)SB);
                // padded rows y0 .. y0 + ROWS of channel m (image rows start P = 16a above)
                for (int l = 0; l < loads; ++l)
                    tma_load_3d(smem + (size_t)s * SB + (size_t)l * box_rows * 128, &ymap, x0, m,
                                y0 + l * box_rows, &full[s]);
                issued = i + 1;
            }
            // every load this CTA issued lands before it may exit (bounded)
            for (int i = (issued > S ? issued - S : 0); i < issued; ++i)
                mbar_wait(&full[i % S], (unsigned)((i / S) & 1));
        }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    // Toeplitz A fragments: A[m][k] = g(16(o - a) + k - m), o = 0..2a
    uint32_t af[2 * A + 1][4];
    {
        const int gm = lane >> 2, tk = (lane & 3) * 2;
        auto tp = [&](int d) { return gs[d < 0 ? -d : d]; };      // |d| <= 16(a+1)
#pragma unroll
        for (int o = 0; o <= 2 * A; ++o) {
            const int base = 16 * (o - A) + tk - gm;
            af[o][0] = Pack<T>::two(tp(base), tp(base + 1));
            af[o][1] = Pack<T>::two(tp(base - 8), tp(base - 7));
            af[o][2] = Pack<T>::two(tp(base + 8), tp(base + 9));
            af[o][3] = Pack<T>::two(tp(base), tp(base + 1));
        }
    }

    // per-thread pixels: warp (rh, cq) owns rows 32rh.. +32, columns 16cq.. +16
    constexpr int RG = KB_ROWS / 32;
    static_assert(KB_CONSUMERS == RG * (KB_COLS / 16), "consumer warps must tile the output tile exactly");
    const int rh = warp % RG, cq = warp / RG;
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

    bool ok = true;
    const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lchunk = 2 * cq + (lane >> 4);
    for (int i = 0; i < C; ++i) {
        const int m = C - 1 - i, s = i % S;
        if (ok && !mbar_wait(&full[s], (unsigned)((i / S) & 1))) {
            ok = false;
            atomicOr(&diag->error_flags, 1u);
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        float acc[2][2][4];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mb][h][e] = 0.0f;
        const unsigned char* st = smem + (size_t)s * SB;
#pragma unroll
        for (int kk = 0; kk < 2 + 2 * A; ++kk) {
            const int row = 16 * (2 * rh + kk) + lrow;
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
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);        // this warp is done with stage s
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e) px[mb][h][e].step(p, m, acc[mb][h][e]);
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

size_t kb_smem_bytes(const TcGeom& g) {
    return (size_t)g.kb_stages * kb_stage_bytes(g.a) + 2 * g.kb_stages * 8 + (16 * (g.a + 1) + 1) * 4 + 1024;
}

template <typename T, int A>
cudaError_t launch_vpass_impl(const float* f, void* Yv, float* out, const GcParams& p, const Taps& t,
                              const TcGeom& g, DiagHeader* diag, cudaStream_t s) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // Y[p][c][x] as a 3-D tensor: x (Wp), c (C), p (Hp); one box = 64 columns x 1 channel x rows
    alignas(64) CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)g.Wp, (cuuint64_t)p.C, (cuuint64_t)g.Hp};
    const cuuint64_t strides[2] = {(cuuint64_t)g.Wp * sizeof(T), (cuuint64_t)p.C * g.Wp * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)KB_COLS, 1u, (cuuint32_t)g.kb_box_rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&map, std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     3, Yv, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = kb_smem_bytes(g);
    auto kern = k_vpass_combine_tc<T, A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.Wp + KB_COLS - 1) / KB_COLS, (g.Hp - 2 * g.P) / KB_ROWS);
    kern<<<grid, 32 * (KB_CONSUMERS + 1), smem, s>>>(map, f, out, p, t, g, diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vpass_a(const float* f, void* Y, float* out, const GcParams& p, const Taps& t, const TcGeom& g,
                           DiagHeader* diag, cudaStream_t s) {
    switch (g.a) {
    case 1: return launch_vpass_impl<T, 1>(f, Y, out, p, t, g, diag, s);
    case 2: return launch_vpass_impl<T, 2>(f, Y, out, p, t, g, diag, s);
    case 3: return launch_vpass_impl<T, 3>(f, Y, out, p, t, g, diag, s);
    case 4: return launch_vpass_impl<T, 4>(f, Y, out, p, t, g, diag, s);
    case 5: return launch_vpass_impl<T, 5>(f, Y, out, p, t, g, diag, s);
    case 6: return launch_vpass_impl<T, 6>(f, Y, out, p, t, g, diag, s);
    case 7: return launch_vpass_impl<T, 7>(f, Y, out, p, t, g, diag, s);
    case 8: return launch_vpass_impl<T, 8>(f, Y, out, p, t, g, diag, s);
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
    // column pass: TMA box of at most 256 rows; stages that fit ~150 KB
    const int rows = kb_tile_rows(g.a);
    g.kb_box_rows = rows <= 256 ? rows : rows / 2;
    g.kb_stages = 4;
    while (g.kb_stages > 2 && (size_t)g.kb_stages * kb_stage_bytes(g.a) > 150 * 1024) --g.kb_stages;
    // tcgen05 row pass
    g.u_tw = g.a <= 4 ? 256 : 64;
    g.u_rows = std::max(1, std::min(128 / std::max(1, C), umma_max_octets() / ((g.u_tw + 32 * g.a) / 8)));
    g.u_hb = (g.a + 3) / 4;
    g.u_nkb = g.u_tw / 64 + 2 * g.u_hb;
    g.u_kbb = (64 + 32 * g.a + 63) / 64;
    return g;
}

size_t tc_workspace_bytes(const TcGeom& g, int C) { return (size_t)C * g.Hp * g.Wp * 2; }

bool tc_supported(int R, int C) {
    if (R > 16 * BF_TC_MAX_A || C > 128) return false;
    const TcGeom g = tc_geometry(64, 64, R, C);
    return umma_smem_bytes(g) <= 227 * 1024 && kb_smem_bytes(g) <= 227 * 1024;
}

cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s) {
    return fp16 ? launch_vpass_a<__half>(f, Y, out, p, t, g, diag, s)
                : launch_vpass_a<__nv_bfloat16>(f, Y, out, p, t, g, diag, s);
}

}  // namespace bfgc
