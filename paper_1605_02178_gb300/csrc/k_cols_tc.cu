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
//                       a tile the ratio and the un-centring into an output tile in shared memory.
// The tile's input pixels arrive by TMA with its first channel pair (the producer loads them once
// every epilogue warp has read the previous tile's), and one thread stores the output tile by
// TMA, so the epilogue issues no global loads or stores on the common path.
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
// The tile's input pixels and output values pass through shared memory as two boxes {32
// columns, 128 rows} of FP32 each (128-byte swizzle: 16-byte chunk c of row r at c ^ (r & 7)),
// loaded and stored by TMA: kPIoBytes for the input tile, as much for the output tile.
constexpr int kPIoBytes = PR * PC * 4;
constexpr int kPIoHalf = kPIoBytes / 2;
// Dynamic shared memory a CTA may use: the 227 KB opt-in limit less the static taps array
// (kTapsSmem floats).
constexpr size_t kPSmemLimit = 227 * 1024 - 4 * 132;

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int c, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n"
                 :: "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(src)) : "memory");
}
// Byte offset of the 16-byte chunk holding columns 4c .. 4c + 3 (c = 0 .. 15) of row r in an
// input or output tile (two 128-byte-swizzled halves of 32 columns)
__device__ __forceinline__ uint32_t io_chunk(int r, int c) {
    return (uint32_t)((c >> 3) * kPIoHalf + r * 128 + (((c & 7) ^ (r & 7)) << 4));
}

}  // namespace

__host__ __device__ inline int vp_rows_in(int a) { return PR + 32 * a; }
__host__ __device__ inline int vp_a_cols(int a) { return vp_rows_in(a) / 2; }
__host__ __device__ inline int vp_bufs(int a) { return (512 - vp_a_cols(a)) / 128; }

// Shared layout (1024-byte aligned): S stages of two channel blocks | input tile | output tile |
// full[S] | empty[S] | tfull[NB] | tempty[NB] | ffull | ffree | TMEM slot | abort flag | last step
// loaded per stage [S] | last step committed per accumulator buffer [NB] | last input tile
// loaded.  Pair step k uses stage k mod S and accumulator buffer k mod NB.  Needs W % 4 == 0 (the
// row pitch of f and out is a TMA stride).
template <typename T, int A_>
__global__ void __launch_bounds__(kPThreads, 1) k_vpass_combine_pairs(
    const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap fmap,
    const __grid_constant__ CUtensorMap omap, const float* __restrict__ f, float* __restrict__ out, const GcParams p,
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
    unsigned char* fs = smem + (size_t)S * SP;                 // input tile (TMA load)
    unsigned char* os = fs + kPIoBytes;                        // output tile (TMA store)
    uint64_t* full = reinterpret_cast<uint64_t*>(os + kPIoBytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NB;
    uint64_t* ffull = tempty + NB;                             // the input tile has landed
    uint64_t* ffree = ffull + 1;                               // every epilogue warp has read it
    uint32_t* tslot = reinterpret_cast<uint32_t*>(ffree + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* stage_k = abort_flag + 1;
    volatile int* buf_j = stage_k + S;
    volatile int* f_last = buf_j + NB;
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
        mbar_init(ffull, 1);
        mbar_init(ffree, kPEpiWarps);
        *f_last = -1;
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
                if (i == 0) {
                    // the tile's input pixels, two boxes {32 columns, 128 rows} of f (zero outside
                    // the image), once every epilogue warp has read the previous tile's
                    if (it > 0 && !mbar_wait_abort(ffree, (unsigned)((it - 1) & 1), abort_flag, diag, kPFlag, p.wait_ns))
                        break;
                    *f_last = it;
                    mbar_expect_tx(ffull, (unsigned)kPIoBytes);
                    tma_load_2d(fs, &fmap, x0, y0, ffull);
                    tma_load_2d(fs + kPIoHalf, &fmap, x0 + 32, y0, ffull);
                }
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
        const uint32_t fsa = su32(fs), osa = su32(os);
        unsigned guarded = 0, illcond = 0;
        bool ok = true;
        auto epi_sync = [] { asm volatile("bar.sync 1, 512;\n" ::: "memory"); };
        int k = 0;
        for (int it = 0; it < my_tiles; ++it) {
            const int tile = (int)blockIdx.x + it * G;
            const int x0 = (tile / tiles_y) * PC, y0 = (tile % tiles_y) * PR;
            const int y = y0 + row, xb = x0 + 16 * cg;
            float u[16], P_[16], Q_[16], Qa[16];
            // this tile's input pixels (TMA): this thread's 16, then the tile is released
            if (ok) {
                bool w = true;
                if (lane == 0) w = mbar_wait_abort(ffull, (unsigned)(it & 1), abort_flag, diag, kPFlag, p.wait_ns);
                ok = __shfl_sync(0xffffffffu, w, 0);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (ok)
                    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(fsa + io_chunk(row, 4 * cg + e)));
                u[4 * e] = v.x; u[4 * e + 1] = v.y; u[4 * e + 2] = v.z; u[4 * e + 3] = v.w;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(ffree);
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
            // eq. (10) into the output tile, which one thread then stores (TMA; clipped to the
            // image).  The tile is free once the previous tile's store has read it.  Pixels the
            // cheap test (ratio_clear) does not clear take the full decision (ratio_decision);
            // guarded or listed ones hold their input value (none of either where the fit
            // converges; the loads of f stay off this path).
            if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
            epi_sync();
            if (ok) {
                unsigned odd = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float o[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int j = 4 * e + h;
                        // 16-bit channels: a 2-ulp quotient (__fdividef) is far below their rounding
                        o[h] = __fdividef(p.s_r * P_[j], Q_[j]) + p.t_c;
                        odd |= (unsigned)(y < p.H && xb + j < p.W && !ratio_clear(p, u[j], P_[j], Q_[j], Qa[j])) << j;
                    }
                    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n"
                                 :: "r"(osa + io_chunk(row, 4 * cg + e)), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3])
                                 : "memory");
                }
                if (__any_sync(0xffffffffu, odd != 0)) {
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
                        if ((redo >> j) & 1u) {
                            const uint32_t a = osa + io_chunk(row, (16 * cg + j) >> 2) + 4 * (j & 3);
                            asm volatile("st.shared.f32 [%0], %1;\n" :: "r"(a), "f"(__ldg(f + i)) : "memory");
                        }
                        refine_push(p, diag, (flag_m >> j) & 1u, (uint32_t)i);
                    }
                }
            }
            // the writes reach the async proxy before the TMA store reads them
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            epi_sync();
            if (tid == 0 && ok) {
                // (x0 < W always; a second half that would start past the image is not stored)
                tma_store_2d(&omap, x0, y0, os);
                if (x0 + 32 < p.W) tma_store_2d(&omap, x0 + 32, y0, os + kPIoHalf);
                asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
            }
        }
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
        count_diag(diag, guarded, illcond);
    }

    // ---- drain: every load issued has landed and every MMA committed has completed (both
    // immediate unless a wait gave up), then release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < S; ++s)
            if (stage_k[s] >= 0) mbar_wait_bounded(&full[s], (unsigned)((stage_k[s] / S) & 1));
        if (*f_last >= 0) mbar_wait_bounded(ffull, (unsigned)(*f_last & 1));
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
    return (size_t)g.vp_stages * 2 * vp_rows_in(g.a) * 128 + 2 * kPIoBytes + (2 * g.vp_stages + 2 * nb + 2) * 8 + 8 +
           4 * (g.vp_stages + nb + 1) + 1024;
}

int vp_stages_for(int a) {
    // channel pairs need two 128-column accumulator buffers beside the Toeplitz operand and at
    // least two stages of two channel tiles beside the input and output tiles
    if (a < 1 || a > 7 || vp_bufs(a) < 2) return 0;        // instantiated for a <= 7
    const size_t stage = (size_t)2 * vp_rows_in(a) * 128;
    int s = 4;
    while (s >= 2 && (size_t)s * stage + 2 * kPIoBytes + 256 + 1024 > kPSmemLimit) --s;
    return s >= 2 ? s : 0;
}

namespace {

// f and out as 2-D FP32 tensors {W, H} with boxes {32, 128} and the 128-byte swizzle (zero fill
// outside the image on loads; stores are clipped to it)
cudaError_t encode_io_map(CUtensorMap* map, const float* ptr, int H, int W) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)W * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)PR};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int A>
cudaError_t launch_pairs_impl(const float* f, void* Yv, float* out, const GcParams& p, const Taps& t,
                              const TcGeom& g, DiagHeader* diag, cudaStream_t s) {
    // one box = 64 columns x 1 channel x kb_box_rows padded rows, 128-byte swizzle
    alignas(64) CUtensorMap map, fmap, omap;
    cudaError_t e = encode_y_map(&map, Yv, g, p.C, std::is_same<T, __half>::value, PC, 1, g.kb_box_rows, true);
    if (e != cudaSuccess) return e;
    if ((e = encode_io_map(&fmap, f, p.H, p.W)) != cudaSuccess) return e;
    if ((e = encode_io_map(&omap, out, p.H, p.W)) != cudaSuccess) return e;
    const size_t smem = vp_smem_bytes(g);
    auto kern = k_vpass_combine_pairs<T, A>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (g.Wp / PC) * ((g.Hp - 2 * g.P) / PR);
    const int grid = std::max(1, std::min(tiles, sms));
    kern<<<grid, kPThreads, smem, s>>>(map, fmap, omap, f, out, p, t, g, diag);
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
