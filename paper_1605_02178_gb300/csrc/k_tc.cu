// Column pass of eq. (7) + ratio (eqs. (8)-(10)) of the fused tensor-core form, on the
// 5th-generation tensor cores (tcgen05), one channel per MMA step: the kernel used when
// ceil(R/16) = 8 (k_cols_tc.cu pairs the channels for smaller radii); and the geometry of the
// fused form.  (The channel build + row pass is k_rows_tc.cu / k_umma.cu.)
//
// GEMM view, per tile of 128 output rows x 64 output columns and per channel m:
//   D[i][x] = sum_k A[i][k] Y_m[y0 + k][x0 + x],   k = 0 .. 128 + 2P - 1  (P = 16a),
//   A[i][k] = g(k - P - i), zero where |k - P - i| > R: the banded Toeplitz matrix of the
//     column Gaussian, 128 x (128 + 32a), held in TENSOR memory for the whole kernel (lane i
//     = row i, 32-bit column c = elements 2c, 2c + 1), so that the MMAs read only B from
//     shared memory;
//   B = the channel's (128 + 32a) x 64 tile of the row-filtered buffer Y, brought in by TMA
//     with the 128-byte swizzle: each 128-byte line holds the 64 columns of one input row,
//     i.e. an MN-major operand (8-row groups 1024 bytes apart);
//   D = 128 tensor-memory lanes x 64 fp32 columns, one of NB accumulator buffers in the
//     tensor-memory columns left over by A.
// 8 + 2a MMAs of 128 x 64 x 16 per tile and channel: 128 + 32a multiply-adds per output,
// against 2R + 1 in the direct sum.  With A in tensor memory an MMA moves 2 KB out of shared
// memory instead of 6 KB (the operand bandwidth of shared memory, 128 bytes per clock, would
// otherwise cost 48 clocks per MMA against 32 of tensor work).
//
// Roles (persistent CTA, one per SM; tiles ordered so that vertically adjacent tiles, which
// share 2P halo rows, run at the same time and meet in L2):
//   warp 16, one lane : TMA producer over an S-stage ring (full / empty mbarriers);
//   warps 17, 18, one lane each : MMA issuers of the even and of the odd channel steps; a
//                       step's MMAs are committed both to the stage's empty barrier (the stage
//                       may be refilled) and to the accumulator buffer's full barrier (the
//                       epilogue may read it).  A thread issuing tcgen05.mma is held for about
//                       45 clocks per 128 x 64 x 16 MMA, so one issuer cannot keep up with the
//                       epilogue and no epilogue warp issues them;
//   warps 0 .. 15     : ratio epilogue, one thread per output row and 16 columns: per channel
//                       one tcgen05.ld of 16 accumulators, then the Horner steps of P, Q and
//                       the guard scale; at the end of a tile the guarded ratio and the
//                       un-centring.  The next tile's input pixels are staged in shared
//                       memory by coalesced cp.async while the current tile runs (registers
//                       are scarce: 19 warps leave 96 per thread).
// Every mbarrier wait is bounded; a wait that runs out flags the workspace and raises a
// shared abort flag that ends the other roles' waits, so the kernel always returns.
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
#include "bfgc_tcgen05.cuh"

namespace bfgc {

using namespace tc;

namespace {

constexpr int VR = 128;                          // output rows per tile (tensor-memory lanes)
constexpr int VC = 64;                           // output columns per tile (MMA N)
constexpr int kEpiWarps = 16;                    // 4 per tensor-memory lane quarter
constexpr int kVThreads = 32 * (kEpiWarps + 3);
constexpr unsigned kVFlag = 1u;                  // error flag of this kernel's waits

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int c, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" :: "r"(su32(dst)), "l"(src) : "memory");
}

}  // namespace

// Input rows of a tile (output rows + halo), tensor-memory columns of A, accumulator buffers
// (an even number: half for the even channel steps, half for the odd ones).
__host__ __device__ inline int vu_rows_in(int a) { return VR + 32 * a; }
__host__ __device__ inline int vu_stage_bytes(int a) { return vu_rows_in(a) * 128; }
__host__ __device__ inline int vu_a_cols(int a) { return vu_rows_in(a) / 2; }
__host__ __device__ inline int vu_bufs(int a) { return (512 - vu_a_cols(a)) / VC / 2 * 2; }
constexpr int kFPitch = VC + 4;                  // floats per row of the staged input tile
constexpr int kFBytes = VR * kFPitch * 4;

// Shared layout (1024-byte aligned): S stages | f tile [128][68] | full[S] | empty[S] |
// tfull[NB] | tempty[NB] | TMEM slot | abort flag | last step loaded per stage [S] | last step
// committed per accumulator buffer [NB].
// Channel step j uses stage (j & 1) S/2 + (j >> 1) mod S/2 and accumulator buffer
// (j & 1) NB/2 + (j >> 1) mod NB/2: even and odd steps have their own stages and buffers, so
// each of the two MMA issuers walks the phases of its barriers in order.
template <typename T, int A_>
__global__ void __launch_bounds__(kVThreads, 1) k_vpass_combine_umma(
    const __grid_constant__ CUtensorMap ymap, const float* __restrict__ f, float* __restrict__ out, const GcParams p,
    const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int RIN = VR + 32 * A_, KS = RIN / 16, SB = RIN * 128;
    constexpr int ACOLS = RIN / 2, NB = (512 - ACOLS) / VC / 2 * 2, NB2 = NB / 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = g.kb_stages, S2 = S / 2, C = p.C, P = g.P;
    const int box_rows = g.kb_box_rows, loads = RIN / box_rows;
    unsigned char* stages = smem;
    float* fs = reinterpret_cast<float*>(smem + (size_t)S * SB);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SB + kFBytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NB;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + NB);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* stage_k = abort_flag + 1;
    volatile int* buf_j = stage_k + S;
    const int tiles_y = (g.Hp - 2 * P) / VR, tiles_x = g.Wp / VC;
    const int ntiles = tiles_x * tiles_y, G = gridDim.x;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const int total = my_tiles * C;                     // channel steps of this CTA
    auto stage_of = [&](int j) { return (j & 1) * S2 + (j >> 1) % S2; };
    auto buf_of = [&](int j) { return (j & 1) * NB2 + (j >> 1) % NB2; };

    __shared__ float s_g[kTapsSmem];
    for (int j = tid; j <= t.R; j += blockDim.x) s_g[j] = t.g[j];
    // ---- set-up: TMEM, barriers
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            stage_k[s] = -1;
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
            buf_j[b] = -1;
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t tacc = tbase + (uint32_t)(512 - NB * VC);         // accumulator buffers

    // ---- the Toeplitz operand into tensor memory: warp q < 4 writes lanes 32q .. 32q + 31
    if (warp < 4) {
        const int i = 32 * warp + lane;
        auto tap = [&](int k) {
            const int d = k - P - i, ad = d < 0 ? -d : d;
            return ad <= t.R ? s_g[ad] : 0.0f;
        };
        for (int c0 = 0; c0 < ACOLS; c0 += 8) {
            uint32_t r[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) r[e] = pack2<T>(tap(2 * (c0 + e)), tap(2 * (c0 + e) + 1));
            tmem_st8(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, r);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    if (warp == kEpiWarps) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            for (int k = 0; k < total; ++k) {
                const int it = k / C, i = k - it * C, s = stage_of(k), use = (k >> 1) / S2;
                const int tile = (int)blockIdx.x + it * G;
                const int x0 = (tile / tiles_y) * VC, y0 = (tile % tiles_y) * VR;
                if (use > 0 && !mbar_wait_abort(&empty[s], (unsigned)((use - 1) & 1), abort_flag, diag, kVFlag, p.wait_ns))
                    break;
                stage_k[s] = k;
                mbar_expect_tx(&full[s], (unsigned)SB);
                // padded rows y0 .. y0 + RIN of channel C-1-i (highest channel first)
                for (int l = 0; l < loads; ++l)
                    tma_load_3d(stages + (size_t)s * SB + (size_t)l * box_rows * 128, &ymap, x0, C - 1 - i,
                                y0 + l * box_rows, &full[s]);
            }
        }
    } else if (warp > kEpiWarps) {
        // ------------------------------------------------------------ MMA issuers (even, odd steps)
        if (lane == 0) {
            // D f32 (bit 4); A, B f16 (0) or bf16 (1) at bits 7, 10; A K-major (bit 15 = 0),
            // B MN-major (bit 16 = 1); N / 8 at bit 17, M / 16 at bit 24
            const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 16) | ((uint32_t)(VC >> 3) << 17) |
                                   ((uint32_t)(VR >> 4) << 24);
            for (int j = warp - kEpiWarps - 1; j < total; j += 2) {
                const int s = stage_of(j), b = buf_of(j);
                const int suse = (j >> 1) / S2, buse = (j >> 1) / NB2;
                if (!mbar_wait_abort(&full[s], (unsigned)(suse & 1), abort_flag, diag, kVFlag, p.wait_ns)) break;
                if (buse > 0 && !mbar_wait_abort(&tempty[b], (unsigned)((buse - 1) & 1), abort_flag, diag, kVFlag, p.wait_ns))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SB), SB);
                const uint32_t d = tacc + (uint32_t)(b * VC);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    // A: 8 tensor-memory columns per k-step; B: 16 lines of 128 bytes per k-step
                    const uint64_t bd = b0 + (uint64_t)(((uint32_t)ks * 16u * 128u) >> 4);
                    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}\n"
                                 :: "r"(d), "r"(tbase + (uint32_t)(8 * ks)), "l"(bd), "r"(idesc),
                                    "r"(ks > 0 ? 1u : 0u));
                }
                buf_j[b] = j;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&empty[s])) : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&tfull[b])) : "memory");
            }
        }
    } else {
        // ------------------------------------------------------------ ratio epilogue
        const int q = warp & 3, cg = warp >> 2;
        const int row = 32 * q + lane;                     // tile-local output row = TMEM lane
        const uint32_t tl = tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * cg);
        const bool vec = (p.W & 3) == 0;
        unsigned guarded = 0, illcond = 0;
        bool ok = true;
        // the tile's 128 x 64 input pixels into fs, 16 bytes per copy, consecutive threads on
        // consecutive addresses (t_c outside the image)
        auto fetch_f = [&](int tile) {
            if (tile >= ntiles) return;
            const int y0 = (tile % tiles_y) * VR, x0 = (tile / tiles_y) * VC;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = tid + 512 * k, r = c >> 4, x = x0 + 4 * (c & 15), y = y0 + r;
                float* dst = fs + r * kFPitch + 4 * (c & 15);
                const float* src = f + (size_t)y * p.W + x;
                if (vec && y < p.H && x + 4 <= p.W) {
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" :: "r"(su32(dst)), "l"(src) : "memory");
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (y < p.H && x + e < p.W) cp_async4(dst + e, src + e);
                        else dst[e] = p.t_c;
                    }
                }
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        };
        auto epi_sync = [] { asm volatile("bar.sync 1, 512;\n" ::: "memory"); };
        fetch_f(blockIdx.x);
        int gi = 0;
        for (int it = 0; it < my_tiles; ++it) {
            const int tile = (int)blockIdx.x + it * G;
            const int y = (tile % tiles_y) * VR + row, xb = (tile / tiles_y) * VC + 16 * cg;
            float u[16], P_[16], Q_[16], Qa[16];
            // this tile's pixels (every warp passes both barriers, also after an abort)
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            epi_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 v = *reinterpret_cast<const float4*>(fs + row * kFPitch + 16 * cg + 4 * k);
                u[4 * k] = v.x; u[4 * k + 1] = v.y; u[4 * k + 2] = v.z; u[4 * k + 3] = v.w;
            }
            epi_sync();
            fetch_f(tile + G);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                u[j] = (u[j] - p.t_c) * p.inv_sr;
                P_[j] = Q_[j] = Qa[j] = 0.0f;
            }
            for (int i = 0; i < C && ok; ++i, ++gi) {
                const int b = buf_of(gi), m = C - 1 - i;
                bool w = true;
                if (lane == 0) w = mbar_wait_abort_poll(&tfull[b], (unsigned)(((gi >> 1) / NB2) & 1), abort_flag, diag, kVFlag, p.wait_ns);
                ok = __shfl_sync(0xffffffffu, w, 0);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                float z[16];
                tmem_ld16(tl + (uint32_t)(b * VC), z);
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
                // Horner steps in u over the filtered channel Z_m (see RatioAcc)
                if (m >= 1) {
                    const float cp = p.coef[m - 1];
#pragma unroll
                    for (int j = 0; j < 16; ++j) P_[j] = fmaf(P_[j], u[j], cp * z[j]);
                }
                if (m <= p.N) {
                    const float cq = p.coef[m];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float qv = cq * z[j];
                        Q_[j] = fmaf(Q_[j], u[j], qv);
                        Qa[j] = fmaf(Qa[j], fabsf(u[j]), fabsf(qv));
                    }
                }
            }
            // eq. (10): every pixel is divided and stored (four at a time); pixels the cheap test
            // (ratio_clear) does not clear take the full decision (ratio_decision) afterwards and,
            // when guarded or listed for the FP64 refinement, are rewritten with their input
            // value (none of either where the fit converges; the loads of f stay off this path).
            if (ok && y < p.H) {
                float* orow = out + (size_t)y * p.W;
                unsigned odd = 0;
#pragma unroll
                for (int j0 = 0; j0 < 16; j0 += 4) {
                    float o[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = j0 + e;
                        // 16-bit channels: a 2-ulp quotient (__fdividef) is far below their rounding
                        o[e] = __fdividef(p.s_r * P_[j], Q_[j]) + p.t_c;
                        odd |= (unsigned)(xb + j < p.W && !ratio_clear(p, u[j], P_[j], Q_[j], Qa[j])) << j;
                    }
                    if (vec && xb + 16 <= p.W) {
                        *reinterpret_cast<float4*>(orow + xb + j0) = make_float4(o[0], o[1], o[2], o[3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (xb + j0 + e < p.W) orow[xb + j0 + e] = o[e];
                    }
                }
                if (__any_sync(__activemask(), odd != 0)) {
                    unsigned redo = 0, flag_m = 0;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if ((odd >> j) & 1u) {
                            const int how = ratio_decision(p, u[j], P_[j], Q_[j], Qa[j]);
                            illcond += how == 1;
                            guarded += how == 2;
                            redo |= (unsigned)(how >= 2) << j;
                            flag_m |= (unsigned)(how == 3) << j;
                        }
                    }
#pragma unroll 1
                    for (int j = 0; j < 16; ++j) {
                        const size_t i = (size_t)y * p.W + xb + j;
                        if ((redo >> j) & 1u) orow[xb + j] = __ldg(f + i);
                        refine_push(p, diag, (flag_m >> j) & 1u, (uint32_t)i);
                    }
                }
            }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        count_diag(diag, guarded, illcond);
    }

    // ---- drain: every load issued has landed and every MMA committed has completed (both
    // immediate unless a wait gave up), then release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < S; ++s)
            if (stage_k[s] >= 0) mbar_wait_bounded(&full[s], (unsigned)(((stage_k[s] >> 1) / S2) & 1));
        for (int b = 0; b < NB; ++b)
            if (buf_j[b] >= 0) mbar_wait_bounded(&tfull[b], (unsigned)(((buf_j[b] >> 1) / NB2) & 1));
    }
    __syncthreads();
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

// ----------------------------------------------------------------------------- host side
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

namespace {

size_t vu_smem_bytes(const TcGeom& g) {
    const int nb = vu_bufs(g.a);
    return (size_t)g.kb_stages * vu_stage_bytes(g.a) + kFBytes + (2 * g.kb_stages + 2 * nb) * 8 + 8 +
           4 * (g.kb_stages + nb) + 1024;
}

template <typename T, int A>
cudaError_t launch_vpass_impl(const float* f, void* Yv, float* out, const GcParams& p, const Taps& t,
                              const TcGeom& g, DiagHeader* diag, cudaStream_t s) {
    // one box = 64 columns x 1 channel x kb_box_rows padded rows, 128-byte swizzle
    alignas(64) CUtensorMap map;
    cudaError_t e = encode_y_map(&map, Yv, g, p.C, std::is_same<T, __half>::value, VC, 1, g.kb_box_rows, true);
    if (e != cudaSuccess) return e;
    const size_t smem = vu_smem_bytes(g);
    auto kern = k_vpass_combine_umma<T, A>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (g.Wp / VC) * ((g.Hp - 2 * g.P) / VR);
    const int grid = std::max(1, std::min(tiles, sms));
    kern<<<grid, kVThreads, smem, s>>>(map, f, out, p, t, g, diag);
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

cudaError_t encode_y_map(CUtensorMap* map, void* Y, const TcGeom& g, int C, bool fp16, int box_x, int box_c,
                         int box_rows, bool swizzle128) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // Y[p][c][x] as a 3-D tensor: x (Wp), c (C), p (Hp)
    const cuuint64_t dims[3] = {(cuuint64_t)g.Wp, (cuuint64_t)C, (cuuint64_t)g.Hp};
    const cuuint64_t strides[2] = {(cuuint64_t)g.Wp * 2, (cuuint64_t)C * g.Wp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_c, (cuuint32_t)box_rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Y, dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

TcGeom tc_geometry(int H, int W, int R, int C, int tw) {
    TcGeom g{};
    g.a = (R + 15) / 16;
    if (g.a < 1) g.a = 1;
    g.P = 16 * g.a;
    g.Hp = (H + VR - 1) / VR * VR + 2 * g.P;
    g.Wp = (W + VC - 1) / VC * VC;
    // column pass: TMA boxes of at most 256 rows; an even number of ring stages (<= 8, half
    // for the even channel steps, half for the odd ones) beside the staged input tile in ~205 KB
    const int rows = vu_rows_in(g.a);
    g.kb_box_rows = rows <= 256 ? rows : rows / 2;
    g.kb_stages = 8;
    while (g.kb_stages > 2 && (size_t)kFBytes + (size_t)g.kb_stages * vu_stage_bytes(g.a) > 205 * 1024)
        g.kb_stages -= 2;
    // tcgen05 row passes (shared-memory Toeplitz; tensor-memory Toeplitz)
    g.u_tw = g.a <= 4 ? (tw == 64 || tw == 128 ? tw : 256) : 64;
    g.u_rows = std::max(1, std::min(128 / std::max(1, C), umma_max_octets() / ((g.u_tw + 32 * g.a) / 8)));
    g.u_hb = (g.a + 3) / 4;
    g.u_nkb = g.u_tw / 64 + 2 * g.u_hb;
    g.u_kbb = (64 + 32 * g.a + 63) / 64;
    g.r_rows = std::max(1, std::min(128 / std::max(1, C), rows_tc_max_octets() / ((128 + 32 * g.a) / 8)));
    // ring depth and staging tiles of the tensor-memory row pass within 224 KB of shared memory
    g.r_np = std::min(128, (g.r_rows * C + 15) / 16 * 16);
    static const int kChoices[8][2] = {{3, 2}, {4, 2}, {3, 3}, {2, 3}, {4, 1}, {3, 1}, {2, 2}, {2, 1}};
    g.vp_stages = vp_stages_for(g.a);
    g.r_stages = 0;
    g.r_stg = 0;
    for (const auto& c : kChoices)
        if ((size_t)c[0] * rows_tc_stage_bytes(g.a, g.r_np) + (size_t)c[1] * rows_tc_stg_bytes(g.r_np) <= 224 * 1024) {
            g.r_stages = c[0];
            g.r_stg = c[1];
            break;
        }
    return g;
}

size_t tc_workspace_bytes(const TcGeom& g, int C) { return (size_t)C * g.Hp * g.Wp * 2; }

bool tc_supported(int R, int C) {
    if (R > 16 * BF_TC_MAX_A || C > 128) return false;
    const TcGeom g = tc_geometry(64, 64, R, C);
    return umma_smem_bytes(g) <= 227 * 1024 && vu_smem_bytes(g) <= 227 * 1024 && vu_bufs(g.a) >= 2 &&
           g.r_stages >= 2 && rows_tc_smem_bytes(g) <= 227 * 1024;
}

cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s) {
    // channel pairs with TMA input / output tiles (rows of f and out a multiple of 16 bytes);
    // otherwise one channel per step
    if (g.vp_stages >= 2 && (p.W & 3) == 0) return launch_vpass_combine_pairs(f, Y, out, p, t, g, fp16, diag, s);
    return fp16 ? launch_vpass_a<__half>(f, Y, out, p, t, g, diag, s)
                : launch_vpass_a<__nv_bfloat16>(f, Y, out, p, t, g, diag, s);
}

}  // namespace bfgc
