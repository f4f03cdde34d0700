// Persistent batched forward of the fused tensor-core form: the row pass (channels of eq. (6)
// after the centring of eq. (17), row half of eq. (7)) and the column pass + ratio (column half
// of eq. (7), eqs. (8)-(10)) of many images, each as ONE launch over a device work list of
// (image, tile) items.
//
// The kernels are those of k_rows_tc.cu and k_cols_tc.cu (same GEMM views, roles and mbarrier
// pipelines) with three changes:
//   * CTA b takes the chunks b, b + grid, ... of the work list (chunks of consecutive items), so
//     that the CTAs work on neighbouring tiles at the same time; every role walks the CTA's items
//     with its own cursor over the images (item0: first item of each image), reloading the
//     image's parameters, tensor maps and pointers from the device table (BatchImg) when it
//     enters the next image of its walk;
//   * every image is laid out at the batch's window block count a (padded rows P = 16a, K of
//     the banded products 128 + 32a) with its own taps, zero beyond its R, so one instantiation
//     serves the whole batch;
//   * the Toeplitz operand is per image: two tensor-memory slots (columns 0 and 128) hold the
//     operands of two consecutive images of the CTA's walk (m-th image: slot m mod 2).  The role
//     that drains the accumulators (row pass: drain warps 0..3; column pass: epilogue warps
//     0..3) writes the operand of image m + 2 into image m's slot once it has waited for the
//     accumulators of image m's last tile (every MMA of image m has completed then), from words
//     packed on the host (BatchImg::tt), and arrives on tready[slot]; the MMA issuer waits there
//     before the first MMA of image m + 2.
// The column pass loads f and stores the output with plain loads and stores (any row pitch).
// Batches with an image whose rows are not 16 bytes long take instantiations (AP) that also
// move whole float2s / float4s inside such rows where their alignment allows;
// the guard of eq. (10) is the FP32 one (no refinement list).  Every wait is bounded.
#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "bfgc_batch.h"
#include "bfgc_common.cuh"
#include "bfgc_tcgen05.cuh"

namespace bfgc {

using namespace tc;

namespace {

// row pass roles (as k_rows_tc.cu)
constexpr int kBDrainWarps = 8;
constexpr int kBGenWarps = 8;
constexpr int kBMmaWarp = kBDrainWarps + kBGenWarps;          // warp 20
constexpr int kBStoreWarp = kBMmaWarp + 1;                    // warp 21
constexpr int kBRowThreads = 32 * (kBStoreWarp + 1);
constexpr int kBGroupWarps = 4;
constexpr int kBGroups = kBGenWarps / kBGroupWarps;
constexpr int kBGroupThreads = 32 * kBGroupWarps;
constexpr int kBOctSlots = 4;
constexpr int kBTile = 128;                                   // output columns per row-pass tile
constexpr int kBN = 128;                                      // product rows (largest of any image)
constexpr uint32_t kBKb = kBN * 128;                          // one 64-column K-block of B
constexpr uint32_t kBStg = kBN * kBTile * 2;                  // one staging tile
// column pass roles (as k_cols_tc.cu)
constexpr int kCRows = 128;                                   // output rows per tile
constexpr int kCCols = 64;                                    // output columns per tile
constexpr int kCEpiWarps = 16;
constexpr int kCThreads = 32 * (kCEpiWarps + 2);
constexpr unsigned kBRowFlag = 4u, kBColFlag = 8u;            // error flags of the two kernels' waits

__device__ __forceinline__ void sts128(uint32_t addr, uint4 w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" :: "r"(addr), "r"(w.x), "r"(w.y), "r"(w.z), "r"(w.w)
                 : "memory");
}
// 16 lanes x 64 columns of tensor memory (fragment layout of 16x256b, as in k_rows_tc.cu)
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
// Four transposed 8x8 matrices of 16-bit values into shared memory, when `on` (warp-uniform)
__device__ __forceinline__ void stmatrix_x4_trans(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                                  uint32_t on) {
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %5, 0;\n"
                 " @q stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};\n}\n"
                 :: "r"(addr), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(on) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int c, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        :: "r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(su32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int c, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n"
                 :: "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(c), "r"(y), "r"(src) : "memory");
}

// The image holding `item`: binary search over the first items (strictly increasing: every
// image has at least one tile)
__device__ __forceinline__ int img_find(const int* __restrict__ item0, int nimg, int item) {
    int l = 0, h = nimg - 1;
    while (l < h) {
        const int m = (l + h + 1) >> 1;
        if (__ldg(item0 + m) <= item) l = m;
        else h = m - 1;
    }
    return l;
}

// A role's cursor over the images of its walk: image `cur` holds items base .. next - 1.
// to(item) moves to the image of a later item and says whether the image changed, so that a
// role reloads its image's parameters only then.
// m counts the images of the walk entered so far (0 for the first).
struct Walk {
    int cur, base, next, m;
    __device__ __forceinline__ void init(const int* __restrict__ item0, int c) {
        cur = c;
        base = __ldg(item0 + c);
        next = __ldg(item0 + c + 1);
        m = 0;
    }
    __device__ __forceinline__ bool to(const int* __restrict__ item0, int item) {
        if (item < next) return false;
        do {
            ++cur;
        } while (__ldg(item0 + cur + 1) <= item);
        base = __ldg(item0 + cur);
        next = __ldg(item0 + cur + 1);
        ++m;
        return true;
    }
};

// The items of CTA b: chunks b, b + G, ... of K consecutive items of the list of w.total
// (b = blockIdx.x, G = gridDim.x); no state beyond the launch's.
template <int K>
struct Items {
    static __device__ __forceinline__ int count(const BatchWork& w) {
        const int b = (int)blockIdx.x, G = (int)gridDim.x, total = w.total;
        const int nchunks = (total + K - 1) / K;
        if (b >= nchunks) return 0;
        const int mine = (nchunks - 1 - b) / G + 1, last = b + (mine - 1) * G;
        return (mine - 1) * K + (last == nchunks - 1 ? total - last * K : K);
    }
    static __device__ __forceinline__ int item(int it) {
        return ((int)blockIdx.x + (it / K) * (int)gridDim.x) * K + it % K;
    }
    // the first item >= x of this CTA (w.total if none)
    static __device__ __forceinline__ int from(const BatchWork& w, int x) {
        const int b = (int)blockIdx.x, G = (int)gridDim.x;
        if (x >= w.total) return w.total;
        const int cx = x / K;
        const int c = cx <= b ? b : b + (cx - b + G - 1) / G * G;
        const int it = c == cx ? x : c * K;
        return it < w.total ? it : w.total;
    }
    // the image of this CTA's walk after image j (nimg if none)
    static __device__ __forceinline__ int next_img(const BatchWork& w, int j) {
        const int x = from(w, __ldg(w.item0 + j + 1));
        return x < w.total ? img_find(w.item0, w.nimg, x) : w.nimg;
    }
};

// The Toeplitz operand of image `im` into tensor-memory columns col .. col + acols - 1 of lane
// quarter q (this warp's): lane i = 32q + l holds A[i][k] = g(k - P - i), zero beyond the
// image's R, as packed 16-bit pairs (column c = elements 2c, 2c + 1), read from the words the
// host packed (BatchImg::tt).  Warp-collective.
__device__ void write_toeplitz(uint32_t col, int q, int lane, const BatchImg* __restrict__ im, int acols) {
    const int i = 32 * q + lane, par = i & 1;
    const uint32_t* __restrict__ src = im->tt[par] + (128 - i - par) / 2;
    for (int c0 = 0; c0 < acols; c0 += 8) {
        uint32_t r[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) r[e] = __ldg(src + c0 + e);
        tmem_st8(col + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// The batch's guard of eq. (10) is the FP32 one of a plan without the refinement
// (clear_rel = 1e-3, no absolute allowance, guard_rel = kGuardRel32): ratio_clear and
// ratio_decision with those parameters, written with them as constants so that no parameter
// is held in registers across the epilogue.
__device__ __forceinline__ bool clear32(float u, float P, float Q, float Qa) {
    return fabsf(u) <= 1.0f && Qa > 0.0f && Qa <= 3.0e38f && fabsf(P) <= 3.0e38f &&
           fabsf(Q) >= (float)kIllcondRel * Qa;
}
__device__ __forceinline__ int decide32(float P, float Q, float Qa) {
    const bool bad = !(Qa > 0.0f) || !(Qa <= 3.0e38f) || !(fabsf(P) <= 3.0e38f);
    if (bad || !(fabsf(Q) >= kGuardRel32 * Qa)) return 2;
    return fabsf(Q) < (float)kIllcondRel * Qa ? 1 : 0;
}

}  // namespace

// ============================================================================= row pass
// Shared layout (1024-byte aligned): S stages of KB K-blocks of 128 rows | NS staging tiles |
// full[S] | empty[S] | dfull[2] | dempty[2] | staged[NS] | freed[NS] | tready[2] | TMEM slot |
// abort flag | last tile committed per accumulator buffer [2].
template <typename T, int A_, bool AP>
__global__ void __launch_bounds__(kBRowThreads, 1) k_rows_batch(const BatchWork w, DiagHeader* diag, int S, int NS) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int KIN = kBTile + 32 * A_, KS = KIN / 16, KB = (KIN + 63) / 64, NO = KIN / 8, PA = 16 * A_;
    constexpr int ACOLS = KIN / 2;
    constexpr uint32_t SB = (uint32_t)KB * kBKb;
    static_assert(ACOLS <= 128, "two Toeplitz slots of 128 columns");
    using I = Items<kBatchRowChunk>;
    const int my_tiles = I::count(w);
    if (my_tiles <= 0) return;                         // the whole CTA, before any set-up
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the first two images of the walk (slots 0 and 1 of the Toeplitz operand)
    const int img_lo = img_find(w.item0, w.nimg, I::item(0)), img_1 = I::next_img(w, img_lo);
    unsigned char* stages = smem;
    unsigned char* stg = smem + (size_t)S * SB;
    uint64_t* full = reinterpret_cast<uint64_t*>(stg + (size_t)NS * kBStg);
    uint64_t* empty = full + S;
    uint64_t* dfull = empty + S;
    uint64_t* dempty = dfull + 2;
    uint64_t* staged = dempty + 2;
    uint64_t* freed = staged + NS;
    uint64_t* tready = freed + NS;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tready + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* last_d = abort_flag + 1;
    const unsigned long long wait_ns = w.wait_ns;

    // ---- build warps: fetch the f values of their first tile before the set-up
    const bool is_build = warp >= kBDrainWarps && warp < kBDrainWarps + kBGenWarps;
    const int NG = min(kBGroups, S);
    const int grp = (warp - kBDrainWarps) / kBGroupWarps;
    const int gtid = tid - 32 * (kBDrainWarps + kBGroupWarps * grp);
    float fv[kBOctSlots][8];
    Walk lw;                                           // image cursor of the fetches and builds
    lw.init(w.item0, img_lo);
    auto load_f = [&](int it) {
#pragma unroll
        for (int s = 0; s < kBOctSlots; ++s)
#pragma unroll
            for (int e = 0; e < 8; ++e) fv[s][e] = 0.0f;
        if (it >= my_tiles) return;
        const int item = I::item(it);
        lw.to(w.item0, item);
        const BatchImg* im = w.imgs + lw.cur;
        const int H = im->p.H, W = im->p.W, TR = im->g.r_rows, Hp = im->g.Hp;
        const int ltx = (im->g.Wp + kBTile - 1) / kBTile;
        const float* __restrict__ f = im->f;
        const int lt = item - lw.base;
        const int ty = lt / ltx, tx = lt - ty * ltx;
        const int p0 = ty * TR, xs0 = tx * kBTile - PA, noct = TR * NO;
        const bool vec = (W & 3) == 0;
#pragma unroll
        for (int s = 0; s < kBOctSlots; ++s) {
            const int o = gtid + s * kBGroupThreads;
            if (o < noct) {
                const int r = o / NO, j = o - r * NO;
                const int pr = p0 + r;
                if (pr < Hp) {
                    int y = pr - PA;
                    y = (unsigned)y < (unsigned)H ? y : mirror(y, H);
                    const float* frow = f + (size_t)y * W;
                    const int xs = xs0 + 8 * j;
                    if (vec && xs >= 0 && xs + 8 <= W) {
                        const float4 a0 = __ldg(reinterpret_cast<const float4*>(frow + xs));
                        const float4 a1 = __ldg(reinterpret_cast<const float4*>(frow + xs + 4));
                        fv[s][0] = a0.x; fv[s][1] = a0.y; fv[s][2] = a0.z; fv[s][3] = a0.w;
                        fv[s][4] = a1.x; fv[s][5] = a1.y; fv[s][6] = a1.z; fv[s][7] = a1.w;
                    } else if (AP && xs >= 0 && xs + 8 <= W && (((size_t)y * W + xs) & 1) == 0) {
                        // (rows not 16-byte aligned) inside the row at an even element: float2s
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            const float2 t = __ldg(reinterpret_cast<const float2*>(frow + xs + e));
                            fv[s][e] = t.x; fv[s][e + 1] = t.y;
                        }
                    } else if (AP && xs >= 0 && xs + 8 <= W) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) fv[s][e] = __ldg(frow + xs + e);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int x = xs + e;
                            fv[s][e] = __ldg(frow + ((unsigned)x < (unsigned)W ? x : mirror(x, W)));
                        }
                    }
                }
            }
        }
    };
    if (is_build && grp < NG) load_f(grp);

    // ---- set-up: TMEM, barriers
    if (warp == kBMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], kBGroupWarps);
            mbar_init(&empty[s], 1);
        }
        for (int d = 0; d < 2; ++d) {
            mbar_init(&dfull[d], 1);
            mbar_init(&dempty[d], kBDrainWarps);
            mbar_init(&tready[d], 4);
            last_d[d] = -1;
        }
        for (int b = 0; b < NS; ++b) {
            mbar_init(&staged[b], kBDrainWarps);
            mbar_init(&freed[b], 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t tacc = tbase + 256u;                // accumulator buffers: columns 256 .. 511
    // the Toeplitz operands of the range's first two images (slots 0 and 1)
    if (warp < 4) {
        write_toeplitz(tbase, warp, lane, w.imgs + img_lo, ACOLS);
        if (img_1 < w.nimg) write_toeplitz(tbase + 128u, warp, lane, w.imgs + img_1, ACOLS);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    if (is_build) {
        // ------------------------------------------------------------ channel build
        // (the fetches run one tile of the group ahead on the same cursor: monotone items)
        auto build = [&](int it) -> bool {
            const int s = it % S, use = it / S;
            if (use > 0 && !mbar_wait_abort(&empty[s], (unsigned)((use - 1) & 1), abort_flag, diag, kBRowFlag, wait_ns))
                return false;
            lw.to(w.item0, I::item(it));
            const BatchImg* im = w.imgs + lw.cur;
            const int C = im->p.C, M = im->g.r_rows * C, NP = im->g.r_np, noct = im->g.r_rows * NO;
            const float t_c = im->p.t_c, inv_sr = im->p.inv_sr, half_mu = im->p.half_mu;
            const uint32_t B = su32(stages + (size_t)s * SB);
            // product rows M .. NP - 1 are read by the MMAs as zeros (an earlier image may have
            // left channels there)
            for (int idx = gtid; idx < (NP - M) * KB * 8; idx += kBGroupThreads) {
                const int row = M + idx / (KB * 8), ch = idx % (KB * 8);
                const int kb = ch >> 3, c16 = ch & 7;
                sts128(B + (uint32_t)kb * kBKb + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
                           (uint32_t)((c16 ^ (row & 7)) << 4),
                       make_uint4(0, 0, 0, 0));
            }
            // channels e u^c of the fetched octets (as k_rows_tc.cu)
#pragma unroll
            for (int sl = 0; sl < kBOctSlots; ++sl) {
                const int o = gtid + sl * kBGroupThreads;
                if (o >= noct) continue;
                const int r = o / NO, j = o - r * NO;
                const int k0 = 8 * j;
                const int chunk = (k0 & 63) >> 3;
                float u[8], e0[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    u[e] = (fv[sl][e] - t_c) * inv_sr;
                    e0[e] = expf(-half_mu * u[e] * u[e]) * ChannelScale<T>::value;
                }
                uint64_t u2[4], v2[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    u2[e] = f2_make(u[2 * e], u[2 * e + 1]);
                    v2[e] = f2_make(e0[2 * e], e0[2 * e + 1]);
                }
                int mrow = r * C;
                const uint32_t Bk = B + (uint32_t)(k0 >> 6) * kBKb;
#pragma unroll 4
                for (int c = 0; c < C; ++c, ++mrow) {
                    uint4 q4;
                    float lo2, hi2;
                    f2_split(v2[0], lo2, hi2); q4.x = pack2<T>(lo2, hi2);
                    f2_split(v2[1], lo2, hi2); q4.y = pack2<T>(lo2, hi2);
                    f2_split(v2[2], lo2, hi2); q4.z = pack2<T>(lo2, hi2);
                    f2_split(v2[3], lo2, hi2); q4.w = pack2<T>(lo2, hi2);
                    sts128(Bk + (uint32_t)mrow * 128u + (uint32_t)((chunk ^ (mrow & 7)) << 4), q4);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v2[e] = f2_mul(v2[e], u2[e]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0 && !(w.stall == 1 && it == 0)) mbar_arrive(&full[s]);
            load_f(it + NG);
            return true;
        };
        if (grp < NG)
            for (int it = grp; it < my_tiles; it += NG)
                if (!build(it)) break;
    } else if (warp == kBMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
            Walk mw;
            mw.init(w.item0, img_lo);
            uint32_t idesc = 0;
            auto mma_enter = [&]() {
                const int NP = w.imgs[mw.cur].g.r_np;
                idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(kBTile >> 4) << 24);
            };
            mma_enter();
            for (int it = 0; it < my_tiles; ++it) {
                const int s = it % S, use = it / S, d = it & 1, duse = it >> 1;
                if (!mbar_wait_abort(&full[s], (unsigned)(use & 1), abort_flag, diag, kBRowFlag, wait_ns)) break;
                // the first tile of the range's image m >= 2: its Toeplitz operand is written
                if (mw.to(w.item0, I::item(it))) {
                    const int m = mw.m;
                    if (m >= 2 && !mbar_wait_abort(&tready[m & 1], (unsigned)(((m - 2) >> 1) & 1), abort_flag, diag,
                                                   kBRowFlag, wait_ns))
                        break;
                    mma_enter();
                }
                const int m = mw.m;
                if (duse > 0 && !mbar_wait_abort(&dempty[d], (unsigned)((duse - 1) & 1), abort_flag, diag, kBRowFlag, wait_ns))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SB));
                const uint32_t dt = tacc + (uint32_t)(d * kBN), ab = tbase + 128u * (uint32_t)(m & 1);
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const uint64_t bd = b0 + (uint64_t)(((uint32_t)(ks >> 2) * kBKb + (uint32_t)(ks & 3) * 32u) >> 4);
                    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}\n"
                                 :: "r"(dt), "r"(ab + (uint32_t)(8 * ks)), "l"(bd), "r"(idesc), "r"(ks > 0 ? 1u : 0u));
                }
                last_d[d] = it;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&empty[s])) : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             :: "r"(su32(&dfull[d])) : "memory");
            }
        }
    } else if (warp == kBStoreWarp) {
        // ------------------------------------------------------------ TMA stores (image's map)
        if (lane == 0) {
            Walk sw;
            sw.init(w.item0, img_lo);
            int TR = 0, Wp = 0, tiles_x = 1;
            const CUtensorMap* map = nullptr;
            auto store_enter = [&]() {
                const BatchImg* im = w.imgs + sw.cur;
                TR = im->g.r_rows;
                Wp = im->g.Wp;
                tiles_x = (Wp + kBTile - 1) / kBTile;
                map = &im->ymap_st;
            };
            store_enter();
            for (int it = 0; it < my_tiles; ++it) {
                const int b = it % NS;
                if (!mbar_wait_abort(&staged[b], (unsigned)((it / NS) & 1), abort_flag, diag, kBRowFlag, wait_ns)) break;
                const int item = I::item(it);
                if (sw.to(w.item0, item)) store_enter();
                const int lt = item - sw.base, ty = lt / tiles_x, tx = lt - ty * tiles_x;
                const uint32_t sb = su32(stg + (size_t)b * kBStg);
                for (int hh = 0; hh < 2; ++hh) {
                    const int xs = tx * kBTile + 64 * hh;
                    if (xs >= Wp) break;
                    tma_store_3d(map, xs, 0, ty * TR, sb + (uint32_t)hh * (kBStg / 2));
                }
                asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
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
        // ------------------------------------------------------------ drain (as k_rows_tc.cu)
        const int q = warp & 3, h = warp >> 2;
        const int mk = lane >> 3, mr = lane & 7;
        auto wait_warp = [&](uint64_t* bar, unsigned parity) {
            bool ok = true;
            if (lane == 0) ok = mbar_wait_abort(bar, parity, abort_flag, diag, kBRowFlag, wait_ns);
            return __shfl_sync(0xffffffffu, ok, 0);
        };
        Walk dw;
        dw.init(w.item0, img_lo);
        int NP = w.imgs[img_lo].g.r_np;
        for (int it = 0; it < my_tiles; ++it) {
            const int d = it & 1, duse = it >> 1, b = it % NS;
            unsigned char* sb = stg + (size_t)b * kBStg;
            if (!wait_warp(&dfull[d], (unsigned)(duse & 1))) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t v0[32], v1[32];
            const uint32_t tl = tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * kBN + 64 * h);
            tmem_ld_16x256b_x8(tl, v0);
            tmem_ld_16x256b_x8(tl + (16u << 16), v1);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&dempty[d]);
            const int item = I::item(it);
            if (dw.to(w.item0, item)) NP = w.imgs[dw.cur].g.r_np;
            const int m = dw.m;
            // the last tile of image m of the walk: every MMA of image m has completed, so its
            // Toeplitz slot takes image m + 2's operand (warps 0..3, one lane quarter each)
            if (h == 0 && it + 1 < my_tiles && I::item(it + 1) >= dw.next) {
                const int j2 = I::next_img(w, img_find(w.item0, w.nimg, I::item(it + 1)));
                if (j2 < w.nimg) {
                    write_toeplitz(tbase + 128u * (uint32_t)(m & 1), q, lane, w.imgs + j2, ACOLS);
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tready[m & 1]);
                }
            }
            if (it >= NS && !wait_warp(&freed[b], (unsigned)((it / NS - 1) & 1))) break;
            auto stage = [&](const uint32_t* v, int L) {
                const int xb = 32 * q + 16 * L + 8 * (mk & 1);
                const uint32_t half = su32(sb) + (uint32_t)(xb >> 6) * (kBStg / 2);
                const int j = (xb & 63) >> 3;
#pragma unroll
                for (int i = 0; i < 8; i += 2) {
                    const int mm = 64 * h + 8 * (i + (mk >> 1)) + mr;
                    const uint32_t addr = half + (uint32_t)mm * 128u + (uint32_t)((j ^ (mm & 7)) << 4);
                    stmatrix_x4_trans(addr,
                                      pack2<T>(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1])),
                                      pack2<T>(__uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3])),
                                      pack2<T>(__uint_as_float(v[4 * i + 4]), __uint_as_float(v[4 * i + 5])),
                                      pack2<T>(__uint_as_float(v[4 * i + 6]), __uint_as_float(v[4 * i + 7])),
                                      64 * h + 8 * i < NP);
                }
            };
            stage(v0, 0);
            stage(v1, 1);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&staged[b]);
        }
    }

    // ---- every MMA committed has completed, then release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int d = 0; d < 2; ++d)
            if (last_d[d] >= 0) mbar_wait_bounded(&dfull[d], (unsigned)((last_d[d] >> 1) & 1));
    }
    __syncthreads();
    if (warp == kBMmaWarp) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

// ============================================================================= column pass
// Shared layout (1024-byte aligned): S stages of two channel blocks | full[S] | empty[S] |
// tfull[2] | tempty[2] | tready[2] | epilogue barrier | TMEM slot | abort flag | last step loaded
// per stage [S] | last step committed per accumulator buffer [2] | the epilogue's image
// parameters and walk.  Pair step k (counted over the CTA's tiles,
// (C + 1) / 2 per tile of an image with C channels) uses stage k mod S and buffer k mod 2.
template <typename T, int A_, bool AP>
__global__ void __launch_bounds__(kCThreads, 1) k_cols_batch(const BatchWork w, DiagHeader* diag, int S) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    constexpr int RIN = kCRows + 32 * A_, KS = RIN / 16, SB = RIN * 128, SP = 2 * SB, PA = 16 * A_;
    constexpr int ACOLS = RIN / 2, NB = 2;
    static_assert(ACOLS <= 128, "two Toeplitz slots of 128 columns");
    using I = Items<kBatchColChunk>;
    const int my_tiles = I::count(w);
    if (my_tiles <= 0) return;                         // the whole CTA, before any set-up
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the first two images of the walk (slots 0 and 1 of the Toeplitz operand)
    const int img_lo = img_find(w.item0, w.nimg, I::item(0)), img_1 = I::next_img(w, img_lo);
    unsigned char* stages = smem;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * SP);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;
    uint64_t* tempty = tfull + NB;
    uint64_t* tready = tempty + NB;
    uint64_t* ebar = tready + 2;                       // the epilogue warps' barrier
    uint32_t* tslot = reinterpret_cast<uint32_t*>(ebar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* stage_k = abort_flag + 1;
    volatile int* buf_j = stage_k + S;
    // the epilogue's copy of the current image's parameters (16-byte aligned)
    GcParams* sp = reinterpret_cast<GcParams*>(
        (reinterpret_cast<uintptr_t>(const_cast<int*>(buf_j + NB)) + 15) & ~(uintptr_t)15);
    int* s_ty = reinterpret_cast<int*>(sp + 1);
    const float** s_f = reinterpret_cast<const float**>(
        (reinterpret_cast<uintptr_t>(s_ty + 1) + 7) & ~(uintptr_t)7);
    float** s_out = reinterpret_cast<float**>(reinterpret_cast<uintptr_t>(s_f + 1));
    int* s_walk = reinterpret_cast<int*>(s_out + 1);          // the epilogue's image: cur, base, next, m
    const unsigned long long wait_ns = w.wait_ns;

    if (warp == kCEpiWarps) {
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
            mbar_init(&tempty[b], kCEpiWarps);
            mbar_init(&tready[b], 4);
            buf_j[b] = -1;
        }
        mbar_init(ebar, kCEpiWarps);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t tacc = tbase + 256u;                // accumulator buffers: columns 256 .. 511
    if (warp < 4) {
        write_toeplitz(tbase, warp, lane, w.imgs + img_lo, ACOLS);
        if (img_1 < w.nimg) write_toeplitz(tbase + 128u, warp, lane, w.imgs + img_1, ACOLS);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    if (warp == kCEpiWarps) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int k = 0;
            bool ok = true;
            Walk pw;
            pw.init(w.item0, img_lo);
            int C = 0, CP = 0, tiles_y = 1, box_rows = 1, loads = 0;
            const CUtensorMap* map = nullptr;
            auto prod_enter = [&]() {
                const BatchImg* im = w.imgs + pw.cur;
                C = im->p.C;
                CP = (C + 1) / 2;
                tiles_y = (im->g.Hp - 2 * PA) / kCRows;
                box_rows = im->g.kb_box_rows;
                loads = RIN / box_rows;
                map = &im->ymap_ld;
            };
            prod_enter();
            for (int it = 0; it < my_tiles && ok; ++it) {
                const int item = I::item(it);
                if (pw.to(w.item0, item)) prod_enter();
                const int lt = item - pw.base;
                const int x0 = (lt / tiles_y) * kCCols, y0 = (lt % tiles_y) * kCRows;
                for (int i = 0; i < CP; ++i, ++k) {
                    const int s = k % S, use = k / S;
                    if (use > 0 && !mbar_wait_abort(&empty[s], (unsigned)((use - 1) & 1), abort_flag, diag, kBColFlag, wait_ns)) {
                        ok = false;
                        break;
                    }
                    if (w.stall == 2 && k == 0) continue;      // (test of the bounded waits)
                    stage_k[s] = k;
                    mbar_expect_tx(&full[s], (unsigned)SP);
                    for (int hh = 0; hh < 2; ++hh) {
                        const int ch = max(C - 1 - 2 * i - hh, 0);
                        for (int l = 0; l < loads; ++l)
                            tma_load_3d(stages + (size_t)s * SP + (size_t)hh * SB + (size_t)l * box_rows * 128, map,
                                        x0, ch, y0 + l * box_rows, &full[s]);
                    }
                }
            }
        }
    } else if (warp == kCEpiWarps + 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (1u << 16) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(kCRows >> 4) << 24);
            int k = 0, mprev = 0;
            bool ok = true;
            Walk mw;
            mw.init(w.item0, img_lo);
            int CP = (w.imgs[img_lo].p.C + 1) / 2;
            for (int it = 0; it < my_tiles && ok; ++it) {
                if (mw.to(w.item0, I::item(it))) CP = (w.imgs[mw.cur].p.C + 1) / 2;
                const int m = mw.m;
                const uint32_t ab = tbase + 128u * (uint32_t)(m & 1);
                for (int i = 0; i < CP; ++i, ++k) {
                    const int s = k % S, use = k / S, b = k % NB, buse = k / NB;
                    ok = mbar_wait_abort_poll(&full[s], (unsigned)(use & 1), abort_flag, diag, kBColFlag, wait_ns);
                    // the first step of the range's image m >= 2: its Toeplitz operand is written
                    if (ok && m != mprev) {
                        if (m >= 2)
                            ok = mbar_wait_abort(&tready[m & 1], (unsigned)(((m - 2) >> 1) & 1), abort_flag, diag,
                                                 kBColFlag, wait_ns);
                        mprev = m;
                    }
                    if (ok && buse > 0)
                        ok = mbar_wait_abort_poll(&tempty[b], (unsigned)((buse - 1) & 1), abort_flag, diag, kBColFlag, wait_ns);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint64_t b0 = sw128_desc(su32(stages + (size_t)s * SP), SB);
                    const uint32_t d = tacc + (uint32_t)(b * 128);
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        const uint64_t bd = b0 + (uint64_t)(((uint32_t)ks * 16u * 128u) >> 4);
                        asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n}\n"
                                     :: "r"(d), "r"(ab + (uint32_t)(8 * ks)), "l"(bd), "r"(idesc), "r"(ks > 0 ? 1u : 0u));
                    }
                    buf_j[b] = k;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                 :: "r"(su32(&empty[s])) : "memory");
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                                 :: "r"(su32(&tfull[b])) : "memory");
                }
            }
        }
    } else {
        // ------------------------------------------------------------ ratio epilogue
        // The current image's parameters live in shared memory (sp), rewritten between two
        // barriers of the 16 epilogue warps when the walk enters the next image, so that no
        // pointer to the table is held across the pair loop.
        const int q = warp & 3, cg = warp >> 2;
        const int row = 32 * q + lane;
        const uint32_t tl = tacc + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * cg);
        bool ok = true;
        // the epilogue warps' barrier: an mbarrier of 16 arrivals with bounded waits (a wait that
        // runs out aborts, as every other wait here)
        unsigned ephase = 0;
        auto epi_sync = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(ebar);
            bool wt = true;
            if (lane == 0) wt = mbar_wait_abort(ebar, ephase & 1u, abort_flag, diag, kBColFlag, wait_ns);
            ++ephase;
            if (!__shfl_sync(0xffffffffu, wt, 0)) ok = false;
        };
        // (the walk's state lives there too: every epilogue thread walks the same items)
        auto epi_enter = [&](int cur, int m) {
            epi_sync();                                // every warp is done with the previous image
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&w.imgs[cur].p);
            uint32_t* dst = reinterpret_cast<uint32_t*>(sp);
            for (int i = tid; i < (int)(sizeof(GcParams) / 4); i += 32 * kCEpiWarps) dst[i] = __ldg(src + i);
            if (tid == 0) {
                *s_ty = (w.imgs[cur].g.Hp - 2 * PA) / kCRows;
                *s_f = w.imgs[cur].f;
                *s_out = w.imgs[cur].out;
                s_walk[0] = cur;
                s_walk[1] = __ldg(w.item0 + cur);
                s_walk[2] = __ldg(w.item0 + cur + 1);
                s_walk[3] = m;
            }
            epi_sync();
        };
        unsigned guarded = 0, illcond = 0;
        int k = 0;
        epi_enter(img_lo, 0);
        const GcParams& p = *sp;
        for (int it = 0; it < my_tiles && ok; ++it) {
            const int item = I::item(it);
            if (item >= s_walk[2]) {
                int cur = s_walk[0];
                do {
                    ++cur;
                } while (__ldg(w.item0 + cur + 1) <= item);
                epi_enter(cur, s_walk[3] + 1);
            }
            const int m = s_walk[3], lt = item - s_walk[1], C = p.C, CP = (C + 1) / 2, tiles_y = *s_ty;
            const int x0 = (lt / tiles_y) * kCCols, y0 = (lt % tiles_y) * kCRows;
            const int y = y0 + row, xb = x0 + 16 * cg;
            const int H = p.H, W = p.W;
            float u[16], P_[16], Q_[16], Qa[16];
            // this thread's 16 input pixels (zero outside the image); converted to u once the
            // first accumulators are in, so that the loads overlap that wait
            {
                const float* __restrict__ f = *s_f;
                if (y < H && (W & 3) == 0 && xb + 16 <= W) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float4 v = __ldg(reinterpret_cast<const float4*>(f + (size_t)y * W + xb) + e);
                        u[4 * e] = v.x; u[4 * e + 1] = v.y; u[4 * e + 2] = v.z; u[4 * e + 3] = v.w;
                    }
                } else if (AP && y < H && xb + 16 <= W) {
                    ldg_run<16>(f, (size_t)y * W + xb, u);             // any 16-byte phase
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) u[j] = (y < H && xb + j < W) ? __ldg(f + (size_t)y * W + xb + j) : 0.0f;
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) P_[j] = Q_[j] = Qa[j] = 0.0f;
            // Horner step in u over the filtered channel Z_m (see RatioAcc)
            auto horner = [&](int mc, const float* z) {
                if (mc >= 1) {
                    const float cp = p.coef[mc - 1];
#pragma unroll
                    for (int j = 0; j < 16; ++j) P_[j] = fmaf(P_[j], u[j], cp * z[j]);
                }
                if (mc <= p.N) {
                    const float cq = p.coef[mc];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float qv = cq * z[j];
                        Q_[j] = fmaf(Q_[j], u[j], qv);
                        Qa[j] = fmaf(Qa[j], fabsf(u[j]), fabsf(qv));
                    }
                }
            };
            for (int i = 0; i < CP; ++i, ++k) {
                const int b = k % NB, m0 = C - 1 - 2 * i;
                bool wt = true;
                if (lane == 0) wt = mbar_wait_abort_poll(&tfull[b], (unsigned)((k / NB) & 1), abort_flag, diag, kBColFlag, wait_ns);
                ok = __shfl_sync(0xffffffffu, wt, 0);
                if (!ok) break;
                if (i == 0) {
                    const float t_c = p.t_c, inv_sr = p.inv_sr;
#pragma unroll
                    for (int j = 0; j < 16; ++j) u[j] = (u[j] - t_c) * inv_sr;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                float z[16];
                tmem_ld16(tl + (uint32_t)(b * 128), z);
                horner(m0, z);
                tmem_ld16(tl + (uint32_t)(b * 128 + 64), z);
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
                if (m0 >= 1) horner(m0 - 1, z);
            }
            if (!ok) break;
            // eq. (10), un-centred; guarded pixels hold their input value.  16-byte (else 8-byte)
            // stores where the row allows them.  The cheap test (ratio_clear) on every pixel and the quotients
            // stored at once; the few pixels it does not clear take the full decision
            // (ratio_decision) afterwards and are rewritten.  (Rows past the image: nothing
            // stored, no pixel odd; the warp vote is taken by all lanes.)
            const float s_r = p.s_r, t_c = p.t_c;
            float* orow = *s_out + (size_t)(y < H ? y : 0) * W;
            unsigned odd = 0;
            if (y < H) {
                // four pixels at a time, stored as they are made (few live registers)
                const bool vec = (W & 3) == 0 && xb + 16 <= W;
                const bool vec2 = AP && !vec && xb + 16 <= W && (((size_t)y * W) & 1) == 0;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float o[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * e + jj;
                        o[jj] = __fdividef(s_r * P_[j], Q_[j]) + t_c;
                        odd |= (unsigned)(xb + j < W && !clear32(u[j], P_[j], Q_[j], Qa[j])) << j;
                    }
                    if (vec) {
                        reinterpret_cast<float4*>(orow + xb)[e] = make_float4(o[0], o[1], o[2], o[3]);
                    } else if (vec2) {
                        reinterpret_cast<float2*>(orow + xb + 4 * e)[0] = make_float2(o[0], o[1]);
                        reinterpret_cast<float2*>(orow + xb + 4 * e)[1] = make_float2(o[2], o[3]);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj)
                            if (xb + 4 * e + jj < W) orow[xb + 4 * e + jj] = o[jj];
                    }
                }
            }
            if (__any_sync(0xffffffffu, odd != 0)) {
                unsigned redo = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if ((odd >> j) & 1u) {
                        const int how = decide32(P_[j], Q_[j], Qa[j]);
                        illcond += how == 1;
                        guarded += how == 2;
                        if (how < 2) orow[xb + j] = s_r * P_[j] / Q_[j] + t_c;
                        redo |= (unsigned)(how >= 2) << j;
                    }
                }
                // guarded pixels: the input value
                const float* frow = *s_f + (size_t)(y < H ? y : 0) * W;
#pragma unroll 1
                for (; redo; redo &= redo - 1) {
                    const int j = __ffs(redo) - 1;
                    orow[xb + j] = __ldg(frow + xb + j);
                }
            }
            // the last tile of image m here: every MMA of image m has completed, so its Toeplitz
            // slot takes image m + 2's operand (warps 0..3, one lane quarter each; after the
            // stores, when no pixel state is live)
            if (cg == 0 && it + 1 < my_tiles && I::item(it + 1) >= s_walk[2]) {
                const int j2 = I::next_img(w, img_find(w.item0, w.nimg, I::item(it + 1)));
                if (j2 < w.nimg) {
                    write_toeplitz(tbase + 128u * (uint32_t)(m & 1), q, lane, w.imgs + j2, ACOLS);
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tready[m & 1]);
                }
            }
        }
        count_diag(diag, guarded, illcond);
    }

    // ---- every load issued has landed and every MMA committed has completed, then release
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < S; ++s)
            if (stage_k[s] >= 0) mbar_wait_bounded(&full[s], (unsigned)((stage_k[s] / S) & 1));
        for (int b = 0; b < NB; ++b)
            if (buf_j[b] >= 0) mbar_wait_bounded(&tfull[b], (unsigned)((buf_j[b] / NB) & 1));
    }
    __syncthreads();
    if (warp == kCEpiWarps) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

// ----------------------------------------------------------------------------- host side
namespace {

size_t rows_stage_bytes(int a) { return (size_t)((kBTile + 32 * a + 63) / 64) * kBKb; }
size_t cols_stage_bytes(int a) { return (size_t)2 * (kCRows + 32 * a) * 128; }
constexpr size_t kBatchSmemLimit = 227 * 1024;

}  // namespace

void rows_batch_ring(int a, int* stages, int* staging) {
    static const int kChoices[6][2] = {{3, 2}, {4, 2}, {3, 3}, {2, 3}, {2, 2}, {2, 1}};
    *stages = *staging = 0;
    for (const auto& c : kChoices)
        if ((size_t)c[0] * rows_stage_bytes(a) + (size_t)c[1] * kBStg <= 224 * 1024) {
            *stages = c[0];
            *staging = c[1];
            return;
        }
}

size_t rows_batch_smem(int a) {
    int S = 0, NS = 0;
    rows_batch_ring(a, &S, &NS);
    return (size_t)S * rows_stage_bytes(a) + (size_t)NS * kBStg + (2 * S + 6 + 2 * NS) * 8 + 32 + 1024;
}

int cols_batch_stages(int a) {
    int s = 4;
    while (s >= 2 && (size_t)s * cols_stage_bytes(a) + 256 + sizeof(GcParams) + 64 + 1024 > kBatchSmemLimit) --s;
    return s >= 2 ? s : 0;
}

size_t cols_batch_smem(int a) {
    const int S = cols_batch_stages(a);
    return (size_t)S * cols_stage_bytes(a) + (2 * S + 7) * 8 + 8 + 4 * (S + 2) + 16 + sizeof(GcParams) + 4 + 8 + 16 +
           16 + 1024;
}

namespace {

template <typename T, int A, bool AP>
cudaError_t rows_impl(const BatchWork& w, int grid, DiagHeader* diag, cudaStream_t s) {
    int S = 0, NS = 0;
    rows_batch_ring(A, &S, &NS);
    if (S < 2) return cudaErrorInvalidValue;
    const size_t smem = rows_batch_smem(A);
    auto kern = k_rows_batch<T, A, AP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBRowThreads, smem, s>>>(w, diag, S, NS);
    return cudaGetLastError();
}

template <typename T, int A, bool AP>
cudaError_t cols_impl(const BatchWork& w, int grid, DiagHeader* diag, cudaStream_t s) {
    const int S = cols_batch_stages(A);
    if (S < 2) return cudaErrorInvalidValue;
    const size_t smem = cols_batch_smem(A);
    auto kern = k_cols_batch<T, A, AP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kCThreads, smem, s>>>(w, diag, S);
    return cudaGetLastError();
}

template <typename T, bool AP>
cudaError_t rows_a(const BatchWork& w, int a, int grid, DiagHeader* diag, cudaStream_t s) {
    switch (a) {
    case 1: return rows_impl<T, 1, AP>(w, grid, diag, s);
    case 2: return rows_impl<T, 2, AP>(w, grid, diag, s);
    case 3: return rows_impl<T, 3, AP>(w, grid, diag, s);
    case 4: return rows_impl<T, 4, AP>(w, grid, diag, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, bool AP>
cudaError_t cols_a(const BatchWork& w, int a, int grid, DiagHeader* diag, cudaStream_t s) {
    switch (a) {
    case 1: return cols_impl<T, 1, AP>(w, grid, diag, s);
    case 2: return cols_impl<T, 2, AP>(w, grid, diag, s);
    case 3: return cols_impl<T, 3, AP>(w, grid, diag, s);
    case 4: return cols_impl<T, 4, AP>(w, grid, diag, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_rows_batch(const BatchWork& w, int a, bool fp16, bool any_pitch, int grid, DiagHeader* diag,
                              cudaStream_t s) {
    if (any_pitch) return fp16 ? rows_a<__half, true>(w, a, grid, diag, s) : rows_a<__nv_bfloat16, true>(w, a, grid, diag, s);
    return fp16 ? rows_a<__half, false>(w, a, grid, diag, s) : rows_a<__nv_bfloat16, false>(w, a, grid, diag, s);
}

cudaError_t launch_cols_batch(const BatchWork& w, int a, bool fp16, bool any_pitch, int grid, DiagHeader* diag,
                              cudaStream_t s) {
    if (any_pitch) return fp16 ? cols_a<__half, true>(w, a, grid, diag, s) : cols_a<__nv_bfloat16, true>(w, a, grid, diag, s);
    return fp16 ? cols_a<__half, false>(w, a, grid, diag, s) : cols_a<__nv_bfloat16, false>(w, a, grid, diag, s);
}

}  // namespace bfgc
