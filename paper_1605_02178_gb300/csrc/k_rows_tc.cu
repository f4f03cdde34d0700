// Channel build + row pass of eq. (7) on the 5th-generation tensor cores (tcgen05), with the
// Toeplitz operand in tensor memory and the output columns on the accumulator lanes.
//
// GEMM view, per tile of 128 output columns (x0 .. x0 + 127) and TR padded rows:
//   D[x][m] = sum_k A[x][k] B[m][k],   k = 0 .. KIN - 1,  KIN = 128 + 32a,
//   A[x][k] = g(k - 16a - x), zero where |k - 16a - x| > R: the banded Toeplitz matrix of the
//     row Gaussian, 128 x KIN, written once into TENSOR memory (lane x, 32-bit column c =
//     elements 2c, 2c + 1), so that the MMAs read only B from shared memory;
//   B[m][k] = the channel e u^c of padded row r at input column x0 - 16a + k, m = r C + c
//     (K-major, 128-byte swizzle, 64-column K-blocks of 128 rows), generated by the CTA from f;
//   D = 128 lanes (output columns) x 128 fp32 columns (product rows m), one of two
//     accumulator buffers.
// 8 + 2a MMAs of 128 x 128 x 16 per tile: 128 + 32a multiply-adds per output and channel.
// An accumulator lane holds one output column for every (row, channel) pair.  Product row m =
// r C + c of the tile is row p0 C + m of Y viewed as Hp C rows of Wp columns, so the whole
// tile is one box {128 columns, C channels, TR padded rows} of the 3-D tensor Y[p][c][x]: the
// drain writes each accumulator column (a product row) into a staging tile [m][x] in shared
// memory, 2 bytes per lane per instruction (a warp fills 64 contiguous bytes), and one thread
// stores the tile with a single TMA bulk tensor store.
//
// Roles (persistent CTA, one per SM, warp-specialised; the phases of a tile meet at mbarriers
// only):
//   warps 8 .. 19 : channel build into an S-stage ring of B buffers (full / empty barriers), in
//                   NG = min(3, S) groups of four warps that take the tiles in turn, so that NG
//                   tiles are built at once (one build thread's power chains are latency-bound);
//                   a group fetches the f values of its next tile into registers while waiting;
//   warp 20, one lane : MMA issuer; a tile's MMAs are committed to the stage's empty barrier
//                   and to the accumulator buffer's full barrier;
//   warps 0 .. 7  : drain, two per tensor-memory lane quarter, 64 product rows each, into
//                   one of NS staging tiles; thread 0 issues the TMA store of the tile.
// Every mbarrier wait is bounded; a wait that runs out flags the workspace and raises a shared
// abort flag that ends the other roles' waits, so the kernel always returns.
#include <cuda.h>

#include <type_traits>

#include "bfgc_common.cuh"
#include "bfgc_tc.h"
#include "bfgc_tcgen05.cuh"

namespace bfgc {

using namespace tc;

namespace {

constexpr int kRDrainWarps = 8;
constexpr int kRGenWarps = 12;
constexpr int kRMmaWarp = kRDrainWarps + kRGenWarps;          // warp 20: MMA issuer
constexpr int kRStoreWarp = kRMmaWarp + 1;                     // warp 21: TMA stores of the tiles
constexpr int kRThreads = 32 * (kRStoreWarp + 1);
constexpr int kRGroupWarps = 4;                   // build groups of four warps (up to three)
constexpr int kRGroups = kRGenWarps / kRGroupWarps;
constexpr int kRGroupThreads = 32 * kRGroupWarps;
constexpr int kROctSlots = 4;                     // 8-column octets per build thread per tile
constexpr int kRTile = 128;                       // output columns per tile (accumulator lanes)
constexpr int kRN = 128;                          // accumulator columns per buffer
// NP = TR C rounded up to 16 (<= 128) product rows per tile (the MMA's N): a K-block of B is NP
// rows of 128 bytes, a staging tile NP rows of 128 columns (two halves of NP 128-byte rows)
constexpr unsigned kRFlag = 4u;                   // error flag of this kernel's waits

// Explicit shared-memory stores (32-bit shared-window addresses), so that no store goes through
// the generic path
__device__ __forceinline__ void sts128(uint32_t addr, uint4 w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" :: "r"(addr), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w)
                 : "memory");
}
__device__ __forceinline__ void sts16(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b16 [%0], %1;\n" :: "r"(addr), "h"((unsigned short)v) : "memory");
}

// 16 lanes x 64 columns of tensor memory, in the fragment layout of 16x256b: thread t holds
// lane t/4 (r[4i], r[4i+1]) and lane t/4 + 8 (r[4i+2], r[4i+3]) at columns 8i + 2(t%4) and
// 8i + 2(t%4) + 1, i = 0 .. 7
__device__ __forceinline__ void tmem_ld_16x256b_x8(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr) : "memory");
}
// Four 8x8 matrices of 16-bit values, stored transposed: smem row i of matrix k (address from
// thread 8k + i) receives column i of the matrix whose row t/4, columns 2(t%4), 2(t%4) + 1 are
// in register k of thread t
// (executed when `on` is non-zero: a warp-uniform predicate, no branch)
__device__ __forceinline__ void stmatrix_x4_trans(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                                  uint32_t on) {
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n"
                 " @q stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};\n}\n"
                 :: "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(on) : "memory");
}

__device__ __forceinline__ void drain_sync() { asm volatile("bar.sync 1, %0;\n" :: "n"(32 * kRDrainWarps) : "memory"); }

}  // namespace

// Shared layout (1024-byte aligned): S stages of KB K-blocks | NS staging tiles | full[S] |
// empty[S] | dfull[2] | dempty[2] | staged[NS] | freed[NS] | TMEM slot | abort flag | last tile
// committed per accumulator buffer [2] | taps [kTapsSmem].
template <typename T, int A_>
__global__ void __launch_bounds__(kRThreads, 1) k_build_hpass_tc(const __grid_constant__ CUtensorMap ymap,
                                                                 const float* __restrict__ f, const GcParams p,
                                                                 const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int a = A_, KIN = kRTile + 32 * A_, KS = KIN / 16, KB = (KIN + 63) / 64, NO = KIN / 8;
    constexpr int ACOLS = KIN / 2;                     // tensor-memory columns of A
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int C = p.C, TR = g.r_rows, S = g.r_stages, NS = g.r_stg, M = TR * C, NP = g.r_np;
    const uint32_t SBk = (uint32_t)NP * 128u, SB = (uint32_t)KB * SBk, STG = (uint32_t)NP * 256u;
    unsigned char* stages = smem;
    unsigned char* stg = smem + (size_t)S * SB;
    uint64_t* full = reinterpret_cast<uint64_t*>(stg + (size_t)NS * STG);
    uint64_t* empty = full + S;
    uint64_t* dfull = empty + S;
    uint64_t* dempty = dfull + 2;
    uint64_t* staged = dempty + 2;                 // staging tile b holds a whole tile (8 drain warps)
    uint64_t* freed = staged + NS;                 // its TMA store has read staging tile b
    uint32_t* tslot = reinterpret_cast<uint32_t*>(freed + NS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* last_d = abort_flag + 1;
    float* s_g = reinterpret_cast<float*>(smem + (size_t)S * SB + (size_t)NS * STG + (2 * S + 4 + 2 * NS) * 8 + 32);
    const int tiles_x = (g.Wp + kRTile - 1) / kRTile, tiles_y = (g.Hp + TR - 1) / TR;
    const int ntiles = tiles_x * tiles_y, G = gridDim.x;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;

    // ---- build warps: the f values of their first tile are fetched before the set-up, so that
    // the loads run while tensor memory, barriers and the Toeplitz operand are prepared
    const bool is_build = warp >= kRDrainWarps && warp < kRDrainWarps + kRGenWarps;
    const int NG = min(kRGroups, S);               // active build groups
    const int grp = (warp - kRDrainWarps) / kRGroupWarps;              // builds tiles grp, grp + NG, ...
    const int gtid = tid - 32 * (kRDrainWarps + kRGroupWarps * grp);   // 0 .. kRGroupThreads - 1
    const int noct = TR * NO;                      // <= kRGroupThreads * kROctSlots (host checks)
    const bool vec = (p.W & 3) == 0;               // 16-byte aligned rows of f
    float fv[kROctSlots][8];
    auto load_f = [&](int tile) {
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int p0 = ty * TR, xs0 = tx * kRTile - 16 * a;
#pragma unroll
        for (int s = 0; s < kROctSlots; ++s) {
            const int o = gtid + s * kRGroupThreads;
#pragma unroll
            for (int e = 0; e < 8; ++e) fv[s][e] = 0.0f;
            if (tile < ntiles && o < noct) {
                const int r = o / NO, j = o - r * NO;
                const int pr = p0 + r;
                if (pr < g.Hp) {
                    int y = pr - g.P;
                    y = (unsigned)y < (unsigned)p.H ? y : mirror(y, p.H);
                    const float* frow = f + (size_t)y * p.W;
                    const int xs = xs0 + 8 * j;
                    if (vec && xs >= 0 && xs + 8 <= p.W) {
                        const float4 a0 = __ldg(reinterpret_cast<const float4*>(frow + xs));
                        const float4 a1 = __ldg(reinterpret_cast<const float4*>(frow + xs + 4));
                        fv[s][0] = a0.x; fv[s][1] = a0.y; fv[s][2] = a0.z; fv[s][3] = a0.w;
                        fv[s][4] = a1.x; fv[s][5] = a1.y; fv[s][6] = a1.z; fv[s][7] = a1.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int x = xs + e;
                            fv[s][e] = __ldg(frow + ((unsigned)x < (unsigned)p.W ? x : mirror(x, p.W)));
                        }
                    }
                }
            }
        }
    };
    if (is_build && grp < NG) load_f((int)blockIdx.x + grp * G);

    // ---- set-up: TMEM, barriers, row table, zero product rows M .. NP - 1 of every stage
    if (warp == kRMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], kRGroupWarps);
            mbar_init(&empty[s], 1);
        }
        for (int d = 0; d < 2; ++d) {
            mbar_init(&dfull[d], 1);
            mbar_init(&dempty[d], kRDrainWarps);
            last_d[d] = -1;
        }
        for (int b = 0; b < NS; ++b) {
            mbar_init(&staged[b], kRDrainWarps);
            mbar_init(&freed[b], 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int j = tid; j <= t.R; j += blockDim.x) s_g[j] = t.g[j];
    for (int idx = tid; idx < S * (NP - M) * KB * 8; idx += blockDim.x) {      // 16-byte chunks
        const int s = idx / ((NP - M) * KB * 8), rem = idx % ((NP - M) * KB * 8);
        const int row = M + rem / (KB * 8), ch = rem % (KB * 8);
        const int kb = ch >> 3, c16 = ch & 7;
        *reinterpret_cast<uint4*>(stages + (size_t)s * SB + (uint32_t)kb * SBk + (row >> 3) * 1024 +
                                  (row & 7) * 128 + ((c16 ^ (row & 7)) << 4)) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t tacc = tbase + 256u;                // accumulator buffers: columns 256 .. 511

    // ---- the Toeplitz operand into tensor memory: warp q < 4 writes lanes 32q .. 32q + 31
    if (warp < 4) {
        const int i = 32 * warp + lane;
        auto tap = [&](int k) {
            const int d = k - 16 * a - i, ad = d < 0 ? -d : d;
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

    if (is_build) {
        // ------------------------------------------------------------ channel build
        // build tile `it` from `fv`, hand it to the MMA issuer, then fetch the group's next tile
        auto build = [&](int it) -> bool {
            const int s = it % S, use = it / S;
            if (use > 0 && !mbar_wait_abort(&empty[s], (unsigned)((use - 1) & 1), abort_flag, diag, kRFlag, p.wait_ns))
                return false;
            unsigned char* B = stages + (size_t)s * SB;
            // channels e u^c of the fetched octets: 8 independent power chains per octet (packed
            // FP32 pairs), one 16-byte shared store per channel
#pragma unroll
            for (int sl = 0; sl < kROctSlots; ++sl) {
                const int o = gtid + sl * kRGroupThreads;
                if (o >= noct) continue;
                const int r = o / NO, j = o - r * NO;
                const int k0 = 8 * j;
                const int chunk = (k0 & 63) >> 3;
                float u[8], e0[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    u[e] = (fv[sl][e] - p.t_c) * p.inv_sr;
                    e0[e] = expf(-p.half_mu * u[e] * u[e]) * ChannelScale<T>::value;
                }
                uint64_t u2[4], v2[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    u2[e] = f2_make(u[2 * e], u[2 * e + 1]);
                    v2[e] = f2_make(e0[2 * e], e0[2 * e + 1]);
                }
                // product row m of a 128-row K-block starts at byte 128 m; its 16-byte chunk
                // `chunk` sits at chunk ^ (m & 7) (128-byte swizzle)
                int mrow = r * C;
                const uint32_t Bk = su32(B) + (uint32_t)(k0 >> 6) * SBk;
#pragma unroll 4
                for (int c = 0; c < C; ++c, ++mrow) {
                    uint4 w;
                    float lo, hi;
                    f2_split(v2[0], lo, hi); w.x = pack2<T>(lo, hi);
                    f2_split(v2[1], lo, hi); w.y = pack2<T>(lo, hi);
                    f2_split(v2[2], lo, hi); w.z = pack2<T>(lo, hi);
                    f2_split(v2[3], lo, hi); w.w = pack2<T>(lo, hi);
                    sts128(Bk + (uint32_t)mrow * 128u + (uint32_t)((chunk ^ (mrow & 7)) << 4), w);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v2[e] = f2_mul(v2[e], u2[e]);
                }
            }
            // one arrive per warp (256 arrives on one barrier would serialise on its word)
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            // (test of the bounded waits, BF_OPT_STALL = 1: the first tile is never handed over;
            // nothing asynchronous is outstanding for it)
            if (lane == 0 && !(p.stall == 1 && it == 0)) mbar_arrive(&full[s]);
            load_f((int)blockIdx.x + (it + NG) * G);
            return true;
        };
        // stage it % S is refilled for tile it after the MMAs of tile it - S; the group's previous
        // wait (tile it - NG) covered tile it - NG - S >= it - 2S, so the phase before the awaited
        // one is complete (NG <= S)
        if (grp < NG)
            for (int it = grp; it < my_tiles; it += NG)
                if (!build(it)) break;
    } else if (warp == kRMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // D f32 (bit 4); A, B f16 (0) or bf16 (1) at bits 7, 10; both K-major (bits 15, 16
            // zero); N / 8 at bit 17, M / 16 at bit 24
            const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NP >> 3) << 17) |
                                   ((uint32_t)(kRTile >> 4) << 24);
            for (int it = 0; it < my_tiles; ++it) {
                const int s = it % S, use = it / S, d = it & 1, duse = it >> 1;
                if (!mbar_wait_abort(&full[s], (unsigned)(use & 1), abort_flag, diag, kRFlag, p.wait_ns)) break;
                if (duse > 0 && !mbar_wait_abort(&dempty[d], (unsigned)((duse - 1) & 1), abort_flag, diag, kRFlag, p.wait_ns))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SB));
                const uint32_t dt = tacc + (uint32_t)(d * kRN);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    // A: 8 tensor-memory columns per k-step; B: 32 bytes per k-step inside a
                    // 64-column K-block, K-blocks SBk apart
                    const uint64_t bd =
                        b0 + (uint64_t)(((uint32_t)(ks >> 2) * SBk + (uint32_t)(ks & 3) * 32u) >> 4);
                    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}\n"
                                 :: "r"(dt), "r"(tbase + (uint32_t)(8 * ks)), "l"(bd), "r"(idesc),
                                    "r"(ks > 0 ? 1u : 0u));
                }
                last_d[d] = it;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&empty[s])) : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&dfull[d])) : "memory");
            }
        }
    } else if (warp == kRStoreWarp) {
        // ------------------------------------------------------------ TMA stores
        // for each tile: wait until the eight drain warps have staged it, store it (two boxes
        // {64 columns, C channels, TR padded rows} from the two 128-byte-swizzled staging halves;
        // rows past Hp and columns past Wp are clipped by the tensor map, a half that starts at or
        // past Wp is skipped), then free the staging tile whose store has been read
        if (lane == 0) {
            for (int it = 0; it < my_tiles; ++it) {
                const int b = it % NS;
                if (!mbar_wait_abort(&staged[b], (unsigned)((it / NS) & 1), abort_flag, diag, kRFlag, p.wait_ns))
                    break;
                const int tile = (int)blockIdx.x + it * G;
                const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
                unsigned char* sb = stg + (size_t)b * STG;
                for (int hh = 0; hh < 2; ++hh) {
                    const int xs = tx * kRTile + 64 * hh;
                    if (xs >= g.Wp) break;
                    asm volatile(
                        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n"
                        :: "l"(reinterpret_cast<uint64_t>(&ymap)), "r"(xs), "r"(0), "r"(ty * TR),
                           "r"(su32(sb) + (uint32_t)hh * (STG / 2))
                        : "memory");
                }
                asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                // free a staging tile once its store has read it.  Two staging tiles: wait for this
                // tile's store (the drain of tile it + 1 fills the other one meanwhile).  Three or
                // more: keep two stores in flight and free the previous tile's (the drain of tile
                // it + NS - 1 waits for it; it has tiles it + 1 .. it + NS - 2 to fill meanwhile)
                if (NS >= 3) {
                    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
                    if (it >= 1) mbar_arrive(&freed[(it - 1) % NS]);
                } else {
                    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
                    mbar_arrive(&freed[b]);
                }
            }
            asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
        }
    } else {
        // ------------------------------------------------------------ drain
        const int q = warp & 3, h = warp >> 2;         // lane quarter, half of the product rows
        // stmatrix row address of this thread: matrix k = lane / 8 covers the 8 columns
        // x = 32q + 16L + 8 (k & 1) .. + 7 and the 8 product rows 64h + 8(i + (k >> 1)) .. + 7
        // of column block pair i; row i8 = lane % 8 of it is 16 bytes of [m][x] in the staging
        // half x / 64 (64 columns, 128-byte rows, 128-byte swizzle: chunk j of row m at
        // j ^ (m & 7))
        const int mk = lane >> 3, mr = lane & 7;
        // each warp on its own: wait for the accumulators (lane 0, bounded; the warp agrees)
        auto wait_warp = [&](uint64_t* bar, unsigned parity) {
            bool w = true;
            if (lane == 0) w = mbar_wait_abort(bar, parity, abort_flag, diag, kRFlag, p.wait_ns);
            return __shfl_sync(0xffffffffu, w, 0);
        };
        for (int it = 0; it < my_tiles; ++it) {
            const int d = it & 1, duse = it >> 1, b = it % NS;
            unsigned char* sb = stg + (size_t)b * STG;
            if (!wait_warp(&dfull[d], (unsigned)(duse & 1))) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // lanes 32q .. 32q + 15 (L = 0) and 32q + 16 .. 32q + 31 (L = 1), columns 64h .. 64h + 63
            uint32_t v0[32], v1[32];
            const uint32_t tl = tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * kRN + 64 * h);
            tmem_ld_16x256b_x8(tl, v0);
            tmem_ld_16x256b_x8(tl + (16u << 16), v1);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[d]);
            // the staging tile's previous store (tile it - NS) has read it
            if (it >= NS && !wait_warp(&freed[b], (unsigned)((it / NS - 1) & 1))) break;
            // product rows m, m + 1 of one column x in one packed conversion; stmatrix with
            // transpose turns the fragments into 16-byte runs of 8 columns of one product row
            // (rows from M on are never stored)
            auto stage = [&](const uint32_t* v, int L) {
                const int xb = 32 * q + 16 * L + 8 * (mk & 1);       // first column of matrix mk
                const uint32_t half = su32(sb) + (uint32_t)(xb >> 6) * (STG / 2);
                const int j = (xb & 63) >> 3;
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const int m = 64 * h + 8 * (i + (mk >> 1)) + mr;
                    const uint32_t addr = half + (uint32_t)m * 128u + (uint32_t)((j ^ (m & 7)) << 4);
                    stmatrix_x4_trans(addr,
                                      pack2<T>(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1])),
                                      pack2<T>(__uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3])),
                                      pack2<T>(__uint_as_float(v[4 * i + 4]), __uint_as_float(v[4 * i + 5])),
                                      pack2<T>(__uint_as_float(v[4 * i + 6]), __uint_as_float(v[4 * i + 7])),
                                      64 * h + 8 * i < NP);           // rows NP .. 127 are not staged
                }
            };
            stage(v0, 0);
            stage(v1, 1);
            // the writes reach the async proxy before the TMA store reads them
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&staged[b]);
        }
    }

    // ---- drain: every MMA committed has completed (immediate unless a wait gave up), then
    // release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int d = 0; d < 2; ++d)
            if (last_d[d] >= 0) mbar_wait_bounded(&dfull[d], (unsigned)((last_d[d] >> 1) & 1));
    }
    __syncthreads();
    if (warp == kRMmaWarp) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

int rows_tc_max_octets() { return kRGroupThreads * kROctSlots; }

size_t rows_tc_stage_bytes(int a, int np) { return (size_t)((kRTile + 32 * a + 63) / 64) * np * 128; }

size_t rows_tc_stg_bytes(int np) { return (size_t)np * kRTile * 2; }

size_t rows_tc_smem_bytes(const TcGeom& g) {
    return (size_t)g.r_stages * rows_tc_stage_bytes(g.a, g.r_np) + (size_t)g.r_stg * rows_tc_stg_bytes(g.r_np) +
           (2 * g.r_stages + 4 + 2 * g.r_stg) * 8 +
           32 + kTapsSmem * 4 + 1024;
}

template <typename T, int A_>
cudaError_t launch_rows_impl(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                             DiagHeader* diag, cudaStream_t s) {
    const size_t smem = rows_tc_smem_bytes(g);
    auto kern = k_build_hpass_tc<T, A_>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the store box of half a tile: 64 columns x C channels x TR padded rows, 128-byte swizzle
    alignas(64) CUtensorMap map;
    e = encode_y_map(&map, Y, g, p.C, std::is_same<T, __half>::value, kRTile / 2, p.C, g.r_rows, true);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.Wp + kRTile - 1) / kRTile) * ((g.Hp + g.r_rows - 1) / g.r_rows);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(tiles, sms));
    kern<<<grid, kRThreads, smem, s>>>(map, f, p, t, g, diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_a(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                          DiagHeader* diag, cudaStream_t s) {
    switch (g.a) {
    case 1: return launch_rows_impl<T, 1>(f, Y, p, t, g, diag, s);
    case 2: return launch_rows_impl<T, 2>(f, Y, p, t, g, diag, s);
    case 3: return launch_rows_impl<T, 3>(f, Y, p, t, g, diag, s);
    case 4: return launch_rows_impl<T, 4>(f, Y, p, t, g, diag, s);
    case 5: return launch_rows_impl<T, 5>(f, Y, p, t, g, diag, s);
    case 6: return launch_rows_impl<T, 6>(f, Y, p, t, g, diag, s);
    case 7: return launch_rows_impl<T, 7>(f, Y, p, t, g, diag, s);
    case 8: return launch_rows_impl<T, 8>(f, Y, p, t, g, diag, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_build_hpass_tc(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                  bool fp16, DiagHeader* diag, cudaStream_t s) {
    return fp16 ? launch_rows_a<__half>(f, Y, p, t, g, diag, s) : launch_rows_a<__nv_bfloat16>(f, Y, p, t, g, diag, s);
}

}  // namespace bfgc
