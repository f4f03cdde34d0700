// Column pass of eq. (7) + ratio (eqs. (8)-(10)) of the fused tensor-core form, two channels
// per MMA step (the kernel used for ceil(R/16) <= 7; k_tc.cu has the one-channel-per-step
// kernel, used beyond).
//
// GEMM view, per tile of 128 output rows x 64 output columns and per pair of channels:
//   D[i][n] = sum_k A[i][k] B[k][n],   k = 0 .. 128 + 2P - 1  (P = 16a),  n = 0 .. 127,
//   A[i][k] = g(k - P - i): the banded Toeplitz matrix of the column Gaussian, 128 x (128 + 32a),
//     held in tensor memory for the whole kernel (lane i = row i, 32-bit column c = elements
//     2c, 2c + 1);
//   B = the (128 + 32a) x 64 tiles of the row-filtered buffer Y of two channels side by side:
//     two 64-column MN blocks (one per channel, one TMA box each, 128-byte swizzle), the
//     second `SB` bytes after the first (the descriptor's leading byte offset);
//   D = 128 tensor-memory lanes x 128 fp32 columns: columns 0 .. 63 the first channel of the
//     pair, 64 .. 127 the second.
// 8 + 2a MMAs of 128 x 128 x 16 per tile and channel pair.  Pairing halves the accumulator
// hand-offs between the MMA issuer and the ratio epilogue (the wait, the tensor-memory load and
// the release are per pair), and one issuing thread keeps up with the epilogue.
//
// Roles (persistent CTA, one per SM; tiles column-major, so that vertically adjacent tiles,
// which share 2P halo rows, run at the same time and meet in L2):
//   warp 16, one lane : TMA producer over an S-stage ring (full / empty mbarriers); a stage
//                       holds one channel pair;
//   warp 17, one lane : MMA issuer; a pair's MMAs are committed to the stage's empty barrier
//                       and to the accumulator buffer's full barrier;
//   warps 0 .. 15     : ratio epilogue, one thread per output row and 16 columns: per pair two
//                       tcgen05.ld of 16 accumulators, each followed by the Horner step of P, Q
//                       and the guard scale for its channel (highest channel first); at the end of
//                       a tile the guarded ratio and the un-centring.  The next tile's input
//                       pixels are staged in shared memory by coalesced cp.async meanwhile.
// With C odd the last pair of a tile repeats channel 0 in its second half, which the epilogue
// ignores.  Every mbarrier wait is bounded; a wait that runs out flags the workspace and raises
// a shared abort flag that ends the other roles' waits, so the kernel always returns.
#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "bfgc_common.cuh"
#include "bfgc_tc.h"
#include "bfgc_tcgen05.cuh"

namespace bfgc {

using namespace tc;

namespace {

constexpr int PR = 128;                          // output rows per tile (tensor-memory lanes)
constexpr int PC = 64;                           // output columns per tile and channel
constexpr int kPEpiWarps = 16;                   // 4 per tensor-memory lane quarter
constexpr int kPThreads = 32 * (kPEpiWarps + 2);
constexpr unsigned kPFlag = 8u;                  // error flag of this kernel's waits
constexpr int kPFPitch = PC + 4;                 // floats per row of the staged input tile
constexpr int kPFBytes = PR * kPFPitch * 4;

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

__host__ __device__ inline int vp_rows_in(int a) { return PR + 32 * a; }
__host__ __device__ inline int vp_a_cols(int a) { return vp_rows_in(a) / 2; }
__host__ __device__ inline int vp_bufs(int a) { return (512 - vp_a_cols(a)) / 128; }

// Shared layout (1024-byte aligned): S stages of two channel blocks | f tile [128][68] |
// full[S] | empty[S] | tfull[NB] | tempty[NB] | TMEM slot | abort flag | last step loaded per
// stage [S] | last step committed per accumulator buffer [NB].  Pair step k uses stage k mod S
// and accumulator buffer k mod NB.
template <typename T, int A_>
__global__ void __launch_bounds__(kPThreads, 1) k_vpass_combine_pairs(
    const __grid_constant__ CUtensorMap ymap, const float* __restrict__ f, float* __restrict__ out, const GcParams p,
    const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int RIN = PR + 32 * A_, KS = RIN / 16, SB = RIN * 128, SP = 2 * SB;
    constexpr int ACOLS = RIN / 2, NB = (512 - ACOLS) / 128;
    static_assert(NB >= 2, "two accumulator buffers of 128 columns");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = g.vp_stages, C = p.C, P = g.P, CP = (C + 1) / 2;
    const int box_rows = g.kb_box_rows, loads = RIN / box_rows;
    unsigned char* stages = smem;
    float* fs = reinterpret_cast<float*>(smem + (size_t)S * SP);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SP + kPFBytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NB;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + NB);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* stage_k = abort_flag + 1;
    volatile int* buf_j = stage_k + S;
    const int tiles_y = (g.Hp - 2 * P) / PR, tiles_x = g.Wp / PC;
    const int ntiles = tiles_x * tiles_y, G = gridDim.x;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const int total = my_tiles * CP;                    // pair steps of this CTA

    __shared__ float s_g[kTapsSmem];
    for (int j = tid; j <= t.R; j += blockDim.x) s_g[j] = t.g[j];
    // ---- set-up: TMEM, barriers
    if (warp == kPEpiWarps) {
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
            mbar_init(&tempty[b], kPEpiWarps);
            buf_j[b] = -1;
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t tacc = tbase + (uint32_t)(512 - NB * 128);        // accumulator buffers

    // ---- the Toeplitz operand into tensor memory: warp q < 4 writes lanes 32q .. 32q + 31.  Only
    // the MMA issuer reads it, so only the writers and the issuer meet on a named barrier (2);
    // the TMA producer and the epilogue's input staging start at once.
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
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        asm volatile("bar.sync 2, 160;\n" ::: "memory");
    }

    if (warp == kPEpiWarps) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            for (int k = 0; k < total; ++k) {
                const int it = k / CP, i = k - it * CP, s = k % S, use = k / S;
                const int tile = (int)blockIdx.x + it * G;
                const int x0 = (tile / tiles_y) * PC, y0 = (tile % tiles_y) * PR;
                if (use > 0 && !mbar_wait_abort(&empty[s], (unsigned)((use - 1) & 1), abort_flag, diag, kPFlag, p.wait_ns))
                    break;
                // (test of the bounded waits, BF_OPT_STALL = 2: the first stage is never loaded;
                // no copy is issued for it)
                if (p.stall == 2 && k == 0) continue;
                stage_k[s] = k;
                mbar_expect_tx(&full[s], (unsigned)SP);
                // padded rows y0 .. y0 + RIN of channels C-1-2i and C-2-2i (channel 0 again when
                // C is odd and the pair runs past it)
                for (int hh = 0; hh < 2; ++hh) {
                    const int ch = max(C - 1 - 2 * i - hh, 0);
                    for (int l = 0; l < loads; ++l)
                        tma_load_3d(stages + (size_t)s * SP + (size_t)hh * SB + (size_t)l * box_rows * 128, &ymap,
                                    x0, ch, y0 + l * box_rows, &full[s]);
                }
            }
        }
    } else if (warp == kPEpiWarps + 1) {
        // ------------------------------------------------------------ MMA issuer
        asm volatile("bar.sync 2, 160;\n" ::: "memory");          // the Toeplitz operand is written
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (lane == 0) {
            // D f32 (bit 4); A, B f16 (0) or bf16 (1) at bits 7, 10; A K-major (bit 15 = 0),
            // B MN-major (bit 16 = 1); N / 8 at bit 17, M / 16 at bit 24
            const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 16) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(PR >> 4) << 24);
            for (int k = 0; k < total; ++k) {
                const int s = k % S, use = k / S, b = k % NB, buse = k / NB;
                if (!mbar_wait_abort_poll(&full[s], (unsigned)(use & 1), abort_flag, diag, kPFlag, p.wait_ns)) break;
                if (buse > 0 && !mbar_wait_abort_poll(&tempty[b], (unsigned)((buse - 1) & 1), abort_flag, diag, kPFlag, p.wait_ns))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // two 64-column MN blocks of B, SB bytes apart (the leading byte offset)
                const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SP), SB);
                const uint32_t d = tacc + (uint32_t)(b * 128);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    // A: 8 tensor-memory columns per k-step; B: 16 lines of 128 bytes per k-step
                    const uint64_t bd = b0 + (uint64_t)(((uint32_t)ks * 16u * 128u) >> 4);
                    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}\n"
                                 :: "r"(d), "r"(tbase + (uint32_t)(8 * ks)), "l"(bd), "r"(idesc),
                                    "r"(ks > 0 ? 1u : 0u));
                }
                buf_j[b] = k;
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
            const int y0 = (tile % tiles_y) * PR, x0 = (tile / tiles_y) * PC;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = tid + 512 * k, r = c >> 4, x = x0 + 4 * (c & 15), y = y0 + r;
                float* dst = fs + r * kPFPitch + 4 * (c & 15);
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
        int k = 0;
        for (int it = 0; it < my_tiles; ++it) {
            const int tile = (int)blockIdx.x + it * G;
            const int y = (tile % tiles_y) * PR + row, xb = (tile / tiles_y) * PC + 16 * cg;
            float u[16], P_[16], Q_[16], Qa[16];
            // this tile's pixels (every warp passes both barriers, also after an abort)
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            epi_sync();
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 v = *reinterpret_cast<const float4*>(fs + row * kPFPitch + 16 * cg + 4 * e);
                u[4 * e] = v.x; u[4 * e + 1] = v.y; u[4 * e + 2] = v.z; u[4 * e + 3] = v.w;
            }
            epi_sync();
            fetch_f(tile + G);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                u[j] = (u[j] - p.t_c) * p.inv_sr;
                P_[j] = Q_[j] = Qa[j] = 0.0f;
            }
            // Horner step in u over the filtered channel Z_m (see RatioAcc)
            auto horner = [&](int m, const float* z) {
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
            };
            for (int i = 0; i < CP && ok; ++i, ++k) {
                const int b = k % NB, m0 = C - 1 - 2 * i;
                bool w = true;
                if (lane == 0) w = mbar_wait_abort_poll(&tfull[b], (unsigned)((k / NB) & 1), abort_flag, diag, kPFlag, p.wait_ns);
                ok = __shfl_sync(0xffffffffu, w, 0);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // the pair's two channels one after the other through one register set; the
                // buffer is released once both are loaded
                float z[16];
                tmem_ld16(tl + (uint32_t)(b * 128), z);
                horner(m0, z);
                tmem_ld16(tl + (uint32_t)(b * 128 + 64), z);
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
                if (m0 >= 1) horner(m0 - 1, z);
            }
            // eq. (10): divided in FP32, guarded, or listed for the FP64 refinement (ratio_decision).
            // Every pixel is stored divided first; the few guarded or listed ones are rewritten
            // with their input value afterwards (the loads of f stay off the common path).
            if (ok && y < p.H) {
                float* orow = out + (size_t)y * p.W;
                float o[16];
                unsigned guard_m = 0, flag_m = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int how = ratio_decision(p, u[j], P_[j], Q_[j], Qa[j]);
                    const bool in = xb + j < p.W;
                    // 16-bit channels: a 2-ulp quotient (__fdividef) is far below their rounding
                    o[j] = __fdividef(p.s_r * P_[j], Q_[j]) + p.t_c;
                    illcond += in && how == 1;
                    guard_m |= (unsigned)(in && how == 2) << j;
                    flag_m |= (unsigned)(in && how == 3) << j;
                }
                if (vec && xb + 16 <= p.W) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(orow + xb + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (xb + j < p.W) orow[xb + j] = o[j];
                }
                // (none of either where the fit converges)
                if (__any_sync(__activemask(), (guard_m | flag_m) != 0)) {
                    guarded += __popc(guard_m);
#pragma unroll 1
                    for (int j = 0; j < 16; ++j)
                        if (((guard_m | flag_m) >> j) & 1u) orow[xb + j] = __ldg(f + (size_t)y * p.W + xb + j);
#pragma unroll 1
                    for (int j = 0; j < 16; ++j)
                        refine_push(p, diag, (flag_m >> j) & 1u, (uint32_t)((size_t)y * p.W + xb + j));
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
            if (stage_k[s] >= 0) mbar_wait_bounded(&full[s], (unsigned)((stage_k[s] / S) & 1));
        for (int b = 0; b < NB; ++b)
            if (buf_j[b] >= 0) mbar_wait_bounded(&tfull[b], (unsigned)((buf_j[b] / NB) & 1));
    }
    __syncthreads();
    if (warp == kPEpiWarps) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

// ----------------------------------------------------------------------------- host side
size_t vp_smem_bytes(const TcGeom& g) {
    const int nb = vp_bufs(g.a);
    return (size_t)g.vp_stages * 2 * vp_rows_in(g.a) * 128 + kPFBytes + (2 * g.vp_stages + 2 * nb) * 8 + 8 +
           4 * (g.vp_stages + nb) + 1024;
}

int vp_stages_for(int a) {
    // channel pairs need two 128-column accumulator buffers beside the Toeplitz operand and at
    // least two stages of two channel tiles beside the staged input tile
    if (a < 1 || a > 8 || vp_bufs(a) < 2) return 0;
    const size_t stage = (size_t)2 * vp_rows_in(a) * 128;
    int s = 4;
    while (s >= 2 && (size_t)s * stage + kPFBytes + 2048 > 224 * 1024) --s;
    return s >= 2 ? s : 0;
}

namespace {

template <typename T, int A>
cudaError_t launch_pairs_impl(const float* f, void* Yv, float* out, const GcParams& p, const Taps& t,
                              const TcGeom& g, DiagHeader* diag, cudaStream_t s) {
    // one box = 64 columns x 1 channel x kb_box_rows padded rows, 128-byte swizzle
    alignas(64) CUtensorMap map;
    cudaError_t e = encode_y_map(&map, Yv, g, p.C, std::is_same<T, __half>::value, PC, 1, g.kb_box_rows, true);
    if (e != cudaSuccess) return e;
    const size_t smem = vp_smem_bytes(g);
    auto kern = k_vpass_combine_pairs<T, A>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (g.Wp / PC) * ((g.Hp - 2 * g.P) / PR);
    const int grid = std::max(1, std::min(tiles, sms));
    kern<<<grid, kPThreads, smem, s>>>(map, f, out, p, t, g, diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pairs_a(const float* f, void* Y, float* out, const GcParams& p, const Taps& t, const TcGeom& g,
                           DiagHeader* diag, cudaStream_t s) {
    switch (g.a) {
    case 1: return launch_pairs_impl<T, 1>(f, Y, out, p, t, g, diag, s);
    case 2: return launch_pairs_impl<T, 2>(f, Y, out, p, t, g, diag, s);
    case 3: return launch_pairs_impl<T, 3>(f, Y, out, p, t, g, diag, s);
    case 4: return launch_pairs_impl<T, 4>(f, Y, out, p, t, g, diag, s);
    case 5: return launch_pairs_impl<T, 5>(f, Y, out, p, t, g, diag, s);
    case 6: return launch_pairs_impl<T, 6>(f, Y, out, p, t, g, diag, s);
    case 7: return launch_pairs_impl<T, 7>(f, Y, out, p, t, g, diag, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_vpass_combine_pairs(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                       const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s) {
    return fp16 ? launch_pairs_a<__half>(f, Y, out, p, t, g, diag, s)
                : launch_pairs_a<__nv_bfloat16>(f, Y, out, p, t, g, diag, s);
}

}  // namespace bfgc
