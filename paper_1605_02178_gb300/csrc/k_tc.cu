// Column pass of eq. (7) + ratio (eqs. (8)-(10)) of the fused tensor-core form, on the
// 5th-generation tensor cores (tcgen05).  (The channel build + row pass is k_umma.cu.)
//
// GEMM view, per tile of 128 output rows x 64 output columns and per channel m:
//   D[i][x] = sum_k A[i][k] Y_m[y0 + k][x0 + x],   k = 0 .. 128 + 2P - 1  (P = 16a),
//   A[i][k] = g(k - P - i), zero where |k - P - i| > R: the banded Toeplitz matrix of the
//     column Gaussian, 128 x (128 + 32a), K-major with the 128-byte swizzle, built once per
//     CTA in shared memory;
//   B = the channel's (128 + 32a) x 64 tile of the row-filtered buffer Y, brought in by TMA
//     with the 128-byte swizzle: each 128-byte line holds the 64 columns of one input row,
//     i.e. an MN-major operand (8-row groups 1024 bytes apart);
//   D = 128 tensor-memory lanes x 64 fp32 columns, one of kTBuf accumulator buffers.
// 8 + 2a MMAs of 128 x 64 x 16 per tile and channel: 128 + 32a multiply-adds per output,
// against 2R + 1 in the direct sum; the tensor cores have the headroom, the kernel is meant
// to be bound by the HBM read of Y.
//
// Schedule (persistent CTA, one per SM; tiles ordered so that vertically adjacent tiles,
// which share 2P halo rows, run at the same time and meet in L2).  A CTA walks its channel
// steps gi = (tile, channel) in order.  All 16 warps run the ratio epilogue, one thread per
// output row and 16 columns: per step one tcgen05.ld of 16 accumulators, then the Horner
// steps of P, Q and the guard scale; at the end of a tile the guarded ratio and the
// un-centring.  The producer and issuer work rotates over the warps: at step gi, one lane
// of warp gi mod 16 issues the MMAs of step gi + LA (committed both to the stage's empty
// barrier and to the accumulator buffer's full barrier) and the TMA load that refills the
// stage freed by the MMAs of an earlier step.  With no warp set aside for it, each SM
// sub-partition holds 4 warps and every thread may use 128 registers.
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

namespace bfgc {

namespace {

constexpr int VR = 128;                          // output rows per tile (tensor-memory lanes)
constexpr int VC = 64;                           // output columns per tile (MMA N)
constexpr int kVWarps = 16;                      // 4 per tensor-memory lane quarter (128 registers)
constexpr int kVThreads = 32 * kVWarps;
constexpr int kTBuf = 8;                         // accumulator buffers of 64 columns (all 512)
constexpr int kLA = 4;                           // MMAs issued up to this many channel steps ahead
constexpr unsigned kVSpin = 1u << 22;            // polls per bounded mbarrier wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(su32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`.  Gives up when another role raised the abort flag, or
// (raising it, and flagging the workspace) when the bounded spin runs out.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                                DiagHeader* diag) {
    for (unsigned i = 0; i < kVSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 31) == 31 && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(&diag->error_flags, 1u);
    return false;
}
// Bounded wait without abort, for draining asynchronous work before the CTA exits.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, unsigned parity) {
    for (unsigned i = 0; i < kVSpin; ++i)
        if (mbar_try_wait(bar, parity)) return;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int c, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(su32(bar))
        : "memory");
}

// Shared-memory matrix descriptor with the 128-byte swizzle: start address, leading and
// stride byte offsets (>> 4), descriptor version 1 (bit 46), swizzle mode 2 (bits 61..63).
// K-major operand: 8-row groups 1024 bytes apart (SBO), LBO unused.  MN-major operand with
// 64 elements per line: 8-line (K) groups 1024 bytes apart (SBO), 64-element MN blocks LBO
// apart (one block here).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr, uint32_t lbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <typename T> __device__ __forceinline__ uint16_t to16(float v);
template <> __device__ __forceinline__ uint16_t to16<__nv_bfloat16>(float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}
template <> __device__ __forceinline__ uint16_t to16<__half>(float v) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* z) {
    uint32_t v[16];
    // load and wait in one statement: the registers are defined only once the wait is done
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) z[j] = __uint_as_float(v[j]);
}

}  // namespace

// Input rows of a tile (output rows + halo) and the shared-memory pieces.
__host__ __device__ inline int vu_rows_in(int a) { return VR + 32 * a; }
__host__ __device__ inline int vu_stage_bytes(int a) { return vu_rows_in(a) * 128; }
__host__ __device__ inline int vu_a_bytes(int a) { return (vu_rows_in(a) + 63) / 64 * VR * 128; }

// Shared layout (1024-byte aligned): Toeplitz A | S stages | full[S] | empty[S] | tfull[kTBuf] |
// tempty[kTBuf] | TMEM slot | abort flag | last channel loaded per stage [S] | last channel
// committed per accumulator buffer [kTBuf].
template <typename T, int A_>
__global__ void __launch_bounds__(kVThreads, 1) k_vpass_combine_umma(
    const __grid_constant__ CUtensorMap ymap, const float* __restrict__ f, float* __restrict__ out, const GcParams p,
    const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int RIN = VR + 32 * A_, KS = RIN / 16, SB = RIN * 128;
    constexpr int KA = (RIN + 63) / 64;                 // 64-column K-blocks of A
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = g.kb_stages, C = p.C, P = g.P;
    const int box_rows = g.kb_box_rows, loads = RIN / box_rows;
    unsigned char* As = smem;
    unsigned char* stages = smem + KA * VR * 128;
    uint64_t* full = reinterpret_cast<uint64_t*>(stages + (size_t)S * SB);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + kTBuf;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + kTBuf);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* stage_k = abort_flag + 1;
    volatile int* buf_j = stage_k + S;
    const int tiles_y = (g.Hp - 2 * P) / VR, tiles_x = g.Wp / VC;
    const int ntiles = tiles_x * tiles_y, G = gridDim.x;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const int total = my_tiles * C;                     // channel steps of this CTA
    // The MMAs of step gi + LA are issued at step gi, the TMA load of step k once the MMAs of
    // step k - S (issued TD steps earlier) are done.  mbarrier waits go by phase parity, so a
    // wait for phase n of a barrier may only start once phase n - 1 is known to be complete:
    // the issuing warp has consumed every step before gi, hence LA < S (full barriers) and
    // LA - TD < S (empty barriers).
    const int LA = S - 1 < kLA ? S - 1 : kLA;
    const int TD = S >= 3 ? 2 : 1;

    // ---- set-up: TMEM, barriers, the Toeplitz operand
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            stage_k[s] = -1;
        }
        for (int b = 0; b < kTBuf; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kVWarps);
            buf_j[b] = -1;
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int idx = tid; idx < VR * KA * 64; idx += blockDim.x) {
        const int i = idx / (KA * 64), k = idx - i * (KA * 64);
        const int d = k - P - i, ad = d < 0 ? -d : d;
        const int kb = k >> 6, kk = k & 63;
        const uint32_t off = (uint32_t)(kb * VR * 128 + (i >> 3) * 1024 + (i & 7) * 128 +
                                        (((kk >> 3) ^ (i & 7)) << 4) + (kk & 7) * 2);
        *reinterpret_cast<uint16_t*>(As + off) = to16<T>(k < RIN && ad <= t.R ? t.g[ad] : 0.0f);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;

    // ---- producer / issuer steps (one lane; any warp may run them)
    // TMA load of channel step k: channel C-1-i of the CTA's tile k / C, padded rows y0 .. y0 + RIN
    auto issue_tma = [&](int k) {
        const int it = k / C, i = k - it * C;
        const int tile = (int)blockIdx.x + it * G;
        const int x0 = (tile / tiles_y) * VC, y0 = (tile % tiles_y) * VR;
        const int s = k % S;
        stage_k[s] = k;
        mbar_expect_tx(&full[s], (unsigned)SB);
        for (int l = 0; l < loads; ++l)
            tma_load_3d(stages + (size_t)s * SB + (size_t)l * box_rows * 128, &ymap, x0, C - 1 - i, y0 + l * box_rows,
                        &full[s]);
    };
    // D f32 (bit 4); A, B f16 (0) or bf16 (1) at bits 7, 10; A K-major (bit 15 = 0), B MN-major
    // (bit 16 = 1); N / 8 at bit 17, M / 16 at bit 24
    const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 16) | ((uint32_t)(VC >> 3) << 17) |
                           ((uint32_t)(VR >> 4) << 24);
    // MMAs of channel step j: stage j % S against the Toeplitz operand into buffer j % kTBuf
    auto issue_mma = [&](int j) -> bool {
        const int s = j % S, b = j % kTBuf;
        if (!mbar_wait_abort(&full[s], (unsigned)((j / S) & 1), abort_flag, diag)) return false;
        if (j >= kTBuf && !mbar_wait_abort(&tempty[b], (unsigned)(((j / kTBuf) - 1) & 1), abort_flag, diag))
            return false;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint64_t a0 = sw128_desc(su32(As), 16);
        const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SB), SB);
        const uint32_t d = tbase + (uint32_t)(b * VC);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            // descriptors advance by adding (byte offset >> 4) to the start address
            const uint64_t ad = a0 + (uint64_t)(((uint32_t)(ks >> 2) * VR * 128u + (uint32_t)(ks & 3) * 32u) >> 4);
            const uint64_t bd = b0 + (uint64_t)(((uint32_t)ks * 16u * 128u) >> 4);
            asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                         :: "r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(ks > 0 ? 1u : 0u));
        }
        buf_j[b] = j;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     :: "r"(su32(&empty[s])) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     :: "r"(su32(&tfull[b])) : "memory");
        return true;
    };
    // the MMAs of channel step c have completed (its stage may be refilled)
    auto mma_done = [&](int c) -> bool {
        return mbar_wait_abort(&empty[c % S], (unsigned)((c / S) & 1), abort_flag, diag);
    };
    // Work of step gi: the MMAs of step gi + LA and the load of step gi + LA + S - TD.  Every
    // wait is on work of an earlier step, so the round-robin over warps cannot deadlock.
    auto control = [&](int gi) -> bool {
        const int j = gi + LA;
        if (j < total && !issue_mma(j)) return false;
        const int k = j + S - TD;
        if (k < total) {
            if (!mma_done(k - S)) return false;
            issue_tma(k);
        }
        return true;
    };

    // ---- prologue (one thread): the loads of steps 0 .. LA + S - TD - 1 and the MMAs of
    // steps 0 .. LA - 1, each MMA after its load (a load past the ring waits for the MMAs of
    // the step that last used its stage)
    if (tid == 0) {
        bool ok = true;
        int next_k = 0;
        auto load_upto = [&](int last) {
            for (; ok && next_k <= last && next_k < total; ++next_k) {
                if (next_k >= S && !(ok = mma_done(next_k - S))) break;
                issue_tma(next_k);
            }
        };
        load_upto(S - 1);
        for (int j = 0; j < LA && j < total && ok; ++j) {
            load_upto(j);
            if (ok) ok = issue_mma(j);
        }
        load_upto(LA + S - TD - 1);
    }
    __syncwarp();

    // ---- ratio epilogue (every warp), one thread per output row and 16 columns
    {
        const int q = warp & 3, cg = warp >> 2;
        const int row = 32 * q + lane;                     // tile-local output row = TMEM lane
        const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * cg);
        const bool vec = (p.W & 3) == 0;
        unsigned guarded = 0, f64 = 0;
        bool ok = true;
        float fv[16];
        auto load_f = [&](int tile) {
            const int y = (tile % tiles_y) * VR + row, xb = (tile / tiles_y) * VC + 16 * cg;
#pragma unroll
            for (int j = 0; j < 16; ++j) fv[j] = p.t_c;
            if (tile < ntiles && y < p.H) {
                const float* fr = f + (size_t)y * p.W;
                if (vec && xb + 16 <= p.W) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        const float4 v = __ldg(reinterpret_cast<const float4*>(fr + xb + j));
                        fv[j] = v.x; fv[j + 1] = v.y; fv[j + 2] = v.z; fv[j + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (xb + j < p.W) fv[j] = __ldg(fr + xb + j);
                }
            }
        };
        load_f(blockIdx.x);
        int gi = 0;
        for (int it = 0; it < my_tiles && ok; ++it) {
            const int tile = (int)blockIdx.x + it * G;
            const int y = (tile % tiles_y) * VR + row, xb = (tile / tiles_y) * VC + 16 * cg;
            float u[16], P_[16], Q_[16], Qa[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                u[j] = (fv[j] - p.t_c) * p.inv_sr;
                P_[j] = Q_[j] = Qa[j] = 0.0f;
            }
            for (int i = 0; i < C; ++i, ++gi) {
                const int b = gi % kTBuf, m = C - 1 - i;
                bool w = true;
                if (lane == 0) {
                    if ((gi & (kVWarps - 1)) == warp) w = control(gi);
                    w = w && mbar_wait_abort(&tfull[b], (unsigned)((gi / kTBuf) & 1), abort_flag, diag);
                }
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
            if (!ok) break;
            if (it + 1 < my_tiles) load_f(tile + G);        // next tile's pixels, in flight meanwhile
            // eq. (10) with the division guard (see RatioAcc::finish), then the store
            if (y < p.H) {
                float o[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (!(fabsf(Q_[j]) >= 1e-12f * Qa[j]) || !(Qa[j] > 0.0f)) {
                        o[j] = xb + j < p.W ? __ldg(f + (size_t)y * p.W + xb + j) : 0.0f;
                        guarded += xb + j < p.W;
                    } else if (fabsf(Q_[j]) < 1e-3f * Qa[j]) {
                        o[j] = (float)((double)p.s_r * (double)P_[j] / (double)Q_[j]) + p.t_c;
                        f64 += xb + j < p.W;
                    } else {
                        o[j] = p.s_r * P_[j] / Q_[j] + p.t_c;
                    }
                }
                float* orow = out + (size_t)y * p.W;
                if (vec && xb + 16 <= p.W) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(orow + xb + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (xb + j < p.W) orow[xb + j] = o[j];
                }
            }
        }
        count_diag(diag, guarded, f64);
    }

    // ---- drain: every load issued has landed and every MMA committed has completed (both
    // immediate unless a wait gave up), then release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < S; ++s)
            if (stage_k[s] >= 0) mbar_drain(&full[s], (unsigned)((stage_k[s] / S) & 1));
        for (int b = 0; b < kTBuf; ++b)
            if (buf_j[b] >= 0) mbar_drain(&tfull[b], (unsigned)((buf_j[b] / kTBuf) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
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

size_t vu_smem_bytes(const TcGeom& g) {
    return (size_t)vu_a_bytes(g.a) + (size_t)g.kb_stages * vu_stage_bytes(g.a) + (2 * g.kb_stages + 2 * kTBuf) * 8 +
           8 + 4 * (g.kb_stages + kTBuf) + 1024;
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
    const cuuint32_t box[3] = {(cuuint32_t)VC, 1u, (cuuint32_t)g.kb_box_rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&map, std::is_same<T, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     3, Yv, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const size_t smem = vu_smem_bytes(g);
    auto kern = k_vpass_combine_umma<T, A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

TcGeom tc_geometry(int H, int W, int R, int C) {
    TcGeom g{};
    g.a = (R + 15) / 16;
    if (g.a < 1) g.a = 1;
    g.P = 16 * g.a;
    g.Hp = (H + VR - 1) / VR * VR + 2 * g.P;
    g.Wp = (W + VC - 1) / VC * VC;
    // column pass: TMA boxes of at most 256 rows; as many ring stages (<= 8) as fit beside
    // the Toeplitz operand in ~200 KB
    const int rows = vu_rows_in(g.a);
    g.kb_box_rows = rows <= 256 ? rows : rows / 2;
    g.kb_stages = 8;
    while (g.kb_stages > 2 && (size_t)vu_a_bytes(g.a) + (size_t)g.kb_stages * vu_stage_bytes(g.a) > 200 * 1024)
        --g.kb_stages;
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
    return umma_smem_bytes(g) <= 227 * 1024 && vu_smem_bytes(g) <= 227 * 1024;
}

cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s) {
    return fp16 ? launch_vpass_a<__half>(f, Y, out, p, t, g, diag, s)
                : launch_vpass_a<__nv_bfloat16>(f, Y, out, p, t, g, diag, s);
}

}  // namespace bfgc
