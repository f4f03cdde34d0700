// Channel build + row pass of eq. (7) on the 5th-generation tensor cores (tcgen05), with the
// Toeplitz operand in shared memory: the variant selected by BF_OPT_TILE_W = 64, 128 or 256
// (the default row pass, k_rows_tc.cu, holds the Toeplitz operand in tensor memory).
//
// GEMM view.  Rows of the product are (padded image row r, channel c) pairs, m = r C + c,
// up to 128 of them per tile (TR = floor(128 / C) padded rows); columns are output columns
// (N = 64 per MMA, TW = 64, 128 or 256 per tile); the contraction runs over input columns.
//   A (128 x K, K-major, 128-byte swizzle, in shared memory): the channels e u^c of the
//     tile's rows over the input columns x0 - 64 HB .. (generated by the CTA from f);
//   B (64 x (64 + 32a), K-major, 128-byte swizzle, shared memory): the banded Toeplitz
//     block B[n][k] = g(k - 16a - n), identical for every 64-column group;
//   D (128 lanes x TW fp32 columns in tensor memory).
// Each 64-column output group uses 4 + 2a k-steps of 16 starting at input column
// 64 HB + 64 g - 16 a (the band), i.e. 64 + 32a multiply-adds per output and channel.
//
// Pipeline (persistent CTA, one per SM; two A buffers, two accumulator buffers):
//   iteration i:  issue the MMAs of tile i+1 (one thread, asynchronous, committed to an
//                 mbarrier) | wait for tile i's MMAs | drain tile i from tensor memory,
//                 staging it in tile i's (now free) A buffer so that every warp store
//                 writes whole 128-byte lines of Y | generate tile i+2's channels into that
//                 A buffer from f values fetched into registers one iteration earlier.
// So the tensor cores work on tile i+1 while the CTA drains tile i and builds tile i+2.
// Every mbarrier wait is bounded; on expiry the kernel flags the workspace and stops.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "bfgc_common.cuh"
#include "bfgc_tc.h"
#include "bfgc_tcgen05.cuh"

namespace bfgc {

using namespace tc;

namespace {

constexpr int kUmmaThreads = 512;                 // 16 warps: 4 per TMEM lane quarter
constexpr int kGenThreads = kUmmaThreads - 32;    // warps 1..15 generate channels
constexpr int kOctSlots = 2;                      // 8-column octets per generator thread per tile

// Byte offset of element (row, k) in a K-major 128-byte-swizzled tile of `rows` rows:
// K-blocks of 64 elements (rows * 128 bytes each), 8-row groups of 1024 bytes, the 16-byte
// chunk j of row r stored at chunk j ^ (r & 7).
__device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
    const int kb = k >> 6, kk = k & 63;
    return (uint32_t)(kb * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 + ((((kk >> 3) ^ (row & 7))) << 4) +
                      (kk & 7) * 2);
}

__device__ __forceinline__ void fence_before_sync_after() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

}  // namespace

// Shared layout (1024-byte aligned): A buffer 0 | A buffer 1 | B | 2 mbarriers | TMEM slot |
// product-row table.
template <typename T, int A_, int TW_>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_build_hpass_umma(const float* __restrict__ f,
                                                                      T* __restrict__ Y, const GcParams p,
                                                                      const Taps t, TcGeom g, DiagHeader* diag) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a, the tile width and the halo blocks are compile-time so that the MMA issue sequence
    // of one thread unrolls into constant descriptor offsets (a single thread issuing
    // tcgen05.mma has no other warps to hide its own address arithmetic behind)
    constexpr int a = A_, TW = TW_, HB = (A_ + 3) / 4;
    static_assert(TW == 64 || TW == 128 || TW == 256, "tile width");
    const int C = p.C, TR = g.u_rows;
    const int M = TR * C;
    const uint32_t a_bytes = (uint32_t)g.u_nkb * 128u * 128u;
    unsigned char* As[2] = {smem, smem + a_bytes};
    unsigned char* Bs = smem + 2 * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + (size_t)g.u_kbb * 64 * 128);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
    int* rowtab = reinterpret_cast<int*>(tslot + 4);   // m -> r * C... as (r << 8) | c, or -1
    const int tiles_x = (g.Wp + TW - 1) / TW, tiles_y = (g.Hp + TR - 1) / TR;
    const int ntiles = tiles_x * tiles_y;
    const int G = gridDim.x;

    // ---- one-time set-up: TMEM, barriers, row table, zero rows M..127 of both A buffers, B
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(su32(&bars[b])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (tid < 128) rowtab[tid] = tid < M ? (((tid / C) << 8) | (tid % C)) : -1;
    for (int idx = tid; idx < 2 * (128 - M) * 64 * g.u_nkb; idx += blockDim.x) {   // 2-byte words
        const int b = idx / ((128 - M) * 64 * g.u_nkb), rem = idx % ((128 - M) * 64 * g.u_nkb);
        const int row = M + rem / (64 * g.u_nkb), k = rem % (64 * g.u_nkb);
        *reinterpret_cast<uint16_t*>(As[b] + sw128_off(row, k, 128)) = 0;
    }
    __shared__ float s_g[kTapsSmem];
    for (int j = tid; j <= t.R; j += blockDim.x) s_g[j] = t.g[j];
    __syncthreads();
    for (int idx = tid; idx < 64 * 64 * g.u_kbb; idx += blockDim.x) {
        const int n = idx / (64 * g.u_kbb), k = idx % (64 * g.u_kbb);
        const int d = k - 16 * a - n;
        const int ad = d < 0 ? -d : d;
        *reinterpret_cast<uint16_t*>(Bs + sw128_off(n, k, 64)) = one16<T>(ad <= t.R ? s_g[ad] : 0.0f);
    }

    // ---- channel generation: every column the MMAs read (the band's k-steps reach 16a
    // beyond the tile on each side; columns past R meet zero taps but must hold finite values)
    const int kgen0 = 64 * HB - 16 * a;                // multiple of 8
    const int NO = (TW + 32 * a) / 8;                  // 8-column octets per padded row
    const int noct = TR * NO;                          // <= kGenThreads * kOctSlots (host checks)
    // Octets (8 consecutive columns of one padded row = one 16-byte chunk of a swizzled row)
    // are owned by the generator threads (warps 1..15), at most kOctSlots each; their f
    // values are fetched into registers an iteration ahead of use.
    const int gtid = tid - 32;
    float fv[kOctSlots][8];
    auto load_f = [&](int tile) {
        const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int p0 = ty * TR, x0 = tx * TW;
#pragma unroll
        for (int s = 0; s < kOctSlots; ++s) {
            const int o = gtid + s * kGenThreads;
#pragma unroll
            for (int e = 0; e < 8; ++e) fv[s][e] = 0.0f;
            if (gtid >= 0 && tile < ntiles && o < noct) {
                const int r = o / NO, j = o - r * NO;
                const int pr = p0 + r;
                if (pr < g.Hp) {
                    int y = pr - g.P;
                    y = (unsigned)y < (unsigned)p.H ? y : mirror(y, p.H);
                    const float* frow = f + (size_t)y * p.W;
                    const int xs = x0 - 64 * HB + kgen0 + 8 * j;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int x = xs + e;
                        fv[s][e] = __ldg(frow + ((unsigned)x < (unsigned)p.W ? x : mirror(x, p.W)));
                    }
                }
            }
        }
    };
    // channels e u^c of the prefetched octets into A: 8 independent power chains per octet,
    // one 16-byte shared store per channel
    auto generate = [&](unsigned char* A) {
#pragma unroll
        for (int s = 0; s < kOctSlots; ++s) {
            const int o = gtid + s * kGenThreads;
            if (gtid < 0 || o >= noct) continue;
            const int r = o / NO, j = o - r * NO;
            const int k0 = kgen0 + 8 * j;
            const uint32_t kbase = (uint32_t)(k0 >> 6) * 128u * 128u;
            const int chunk = (k0 & 63) >> 3;
            float u[8], v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                u[e] = (fv[s][e] - p.t_c) * p.inv_sr;
                v[e] = expf(-p.half_mu * u[e] * u[e]) * ChannelScale<T>::value;
            }
            int mrow = r * C;
            for (int c = 0; c < C; ++c, ++mrow) {
                const uint32_t off = kbase + (uint32_t)(mrow >> 3) * 1024u + (uint32_t)(mrow & 7) * 128u +
                                     (uint32_t)((chunk ^ (mrow & 7)) << 4);
                uint4 w;
                w.x = pack2<T>(v[0], v[1]);
                w.y = pack2<T>(v[2], v[3]);
                w.z = pack2<T>(v[4], v[5]);
                w.w = pack2<T>(v[6], v[7]);
                *reinterpret_cast<uint4*>(A + off) = w;
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] *= u[e];
            }
        }
    };

    // instruction descriptor: D f32 (bit 4), A and B f16 (0) or bf16 (1) at bits 7 and 10,
    // both K-major, N / 8 at bit 17, M / 16 at bit 24
    const uint32_t fmt = std::is_same<T, __half>::value ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
    uint32_t tbase = 0;
    // MMAs of `tile` from A buffer `buf` into accumulator buffer `buf` (thread 0 only)
    auto issue_mma = [&](int buf) {
        const uint64_t a0 = sw128_desc(su32(As[buf])), b0 = sw128_desc(su32(Bs));
        const uint32_t d0 = tbase + (uint32_t)(buf * TW);
#pragma unroll
        for (int gi = 0; gi < TW / 64; ++gi) {
#pragma unroll
            for (int j = 0; j < 4 + 2 * a; ++j) {
                const int ks = 4 * HB + 4 * gi - a + j;
                // descriptors advance by adding (byte offset >> 4) to the start-address field;
                // with everything unrolled these offsets are constants
                const uint64_t ad = a0 + (uint64_t)(((uint32_t)(ks >> 2) * 128u * 128u + (uint32_t)(ks & 3) * 32u) >> 4);
                const uint64_t bd = b0 + (uint64_t)(((uint32_t)(j >> 2) * 64u * 128u + (uint32_t)(j & 3) * 32u) >> 4);
                asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n"
                             :: "r"(d0 + 64u * gi), "l"(ad), "l"(bd), "r"(idesc), "r"(j > 0 ? 1u : 0u));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                     :: "r"(su32(&bars[buf])) : "memory");
    };

    // epilogue geometry: warp (lane quarter q, column slot cw); ncw column slots of cpw columns
    const int q = warp & 3;
    const int ncw = TW >= 128 ? 4 : TW / 32;
    const int cw = warp >> 2;
    const int cpw = TW / ncw;                          // 64 (TW = 256) or 32 (TW = 128, 64)
    const int spitch = cpw * 2 + 16;                   // staging row pitch (bytes)
    const int lpr = cpw / 8;                           // 16-byte chunks per staged row: 8 or 4

    // ---- prologue: tiles t0 and t0+G generated, MMAs of t0 issued
    int tile = blockIdx.x;
    load_f(tile);
    generate(As[0]);
    load_f(tile + G);
    fence_before_sync_after();
    tbase = *tslot;
    if (tid == 0 && tile < ntiles) issue_mma(0);
    if (tile + G < ntiles) generate(As[1]);
    load_f(tile + 2 * G);
    fence_before_sync_after();
    bool ok = true;

    for (int it = 0; tile < ntiles; ++it, tile += G) {
        const int b = it & 1;
        if (tid == 0 && ok && tile + G < ntiles) issue_mma(b ^ 1);     // tile + G, already generated

        // drain tile `tile` (accumulators b), staged through A buffer b
        if (ok && !mbar_wait_bounded(&bars[b], (unsigned)((it >> 1) & 1))) {
            ok = false;
            atomicOr(&diag->error_flags, 2u);
        }
        ok = __all_sync(0xffffffffu, ok);              // tcgen05.ld below is warp-collective
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (ok && cw < ncw) {
            const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
            const int p0 = ty * TR, x0 = tx * TW;
            unsigned char* stg = As[b] + (size_t)warp * 32 * spitch;
            for (int c0 = 0; c0 < cpw; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * TW + cw * cpw + c0), v);
                uint4* srow = reinterpret_cast<uint4*>(stg + lane * spitch + c0 * 2);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint4 w;
                    w.x = pack2<T>(__uint_as_float(v[8 * k + 0]), __uint_as_float(v[8 * k + 1]));
                    w.y = pack2<T>(__uint_as_float(v[8 * k + 2]), __uint_as_float(v[8 * k + 3]));
                    w.z = pack2<T>(__uint_as_float(v[8 * k + 4]), __uint_as_float(v[8 * k + 5]));
                    w.w = pack2<T>(__uint_as_float(v[8 * k + 6]), __uint_as_float(v[8 * k + 7]));
                    srow[k] = w;
                }
            }
            __syncwarp();
            // each store instruction writes 32 / lpr whole rows of cpw columns
            const int rows_per_step = 32 / lpr;
            const int xcol = x0 + cw * cpw + (lane % lpr) * 8;
            for (int r0 = 0; r0 < 32; r0 += rows_per_step) {
                const int rr = r0 + lane / lpr;
                const int info = rowtab[32 * q + rr];
                const int pr = p0 + (info >> 8);
                if (info >= 0 && pr < g.Hp && xcol < g.Wp) {
                    const uint4 w = *reinterpret_cast<const uint4*>(stg + rr * spitch + (lane % lpr) * 16);
                    *reinterpret_cast<uint4*>(Y + ((size_t)pr * C + (info & 255)) * g.Wp + xcol) = w;
                }
            }
        }
        __syncthreads();                               // staging reads done before A buffer b is rebuilt
        if (tile + 2 * G < ntiles) generate(As[b]);    // tile + 2G
        load_f(tile + 3 * G);
        fence_before_sync_after();
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tbase), "r"(512));
    }
}

int umma_max_octets() { return kGenThreads * kOctSlots; }

size_t umma_smem_bytes(const TcGeom& g) {
    return (size_t)2 * g.u_nkb * 128 * 128 + (size_t)g.u_kbb * 64 * 128 + 64 + 128 * 4 + 1024;
}

template <typename T, int A_, int TW_>
cudaError_t launch_umma_impl(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                             DiagHeader* diag, cudaStream_t s, int grid, size_t smem) {
    auto kern = k_build_hpass_umma<T, A_, TW_>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kUmmaThreads, smem, s>>>(f, static_cast<T*>(Y), p, t, g, diag);
    return cudaGetLastError();
}

// a <= 4: tile widths 64, 128 and 256; a > 4 (two 64-column halo blocks a side): 64 only
template <typename T, int A_>
cudaError_t launch_umma_tw(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                           DiagHeader* diag, cudaStream_t s, int grid, size_t smem) {
    if constexpr (A_ <= 4) {
        if (g.u_tw == 256) return launch_umma_impl<T, A_, 256>(f, Y, p, t, g, diag, s, grid, smem);
        if (g.u_tw == 128) return launch_umma_impl<T, A_, 128>(f, Y, p, t, g, diag, s, grid, smem);
    }
    if (g.u_tw == 64) return launch_umma_impl<T, A_, 64>(f, Y, p, t, g, diag, s, grid, smem);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_umma_a(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                          DiagHeader* diag, cudaStream_t s, int grid, size_t smem) {
    switch (g.a) {
    case 1: return launch_umma_tw<T, 1>(f, Y, p, t, g, diag, s, grid, smem);
    case 2: return launch_umma_tw<T, 2>(f, Y, p, t, g, diag, s, grid, smem);
    case 3: return launch_umma_tw<T, 3>(f, Y, p, t, g, diag, s, grid, smem);
    case 4: return launch_umma_tw<T, 4>(f, Y, p, t, g, diag, s, grid, smem);
    case 5: return launch_umma_tw<T, 5>(f, Y, p, t, g, diag, s, grid, smem);
    case 6: return launch_umma_tw<T, 6>(f, Y, p, t, g, diag, s, grid, smem);
    case 7: return launch_umma_tw<T, 7>(f, Y, p, t, g, diag, s, grid, smem);
    case 8: return launch_umma_tw<T, 8>(f, Y, p, t, g, diag, s, grid, smem);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_build_hpass_umma(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                    bool fp16, DiagHeader* diag, cudaStream_t s) {
    const size_t smem = umma_smem_bytes(g);
    const int tiles = ((g.Wp + g.u_tw - 1) / g.u_tw) * ((g.Hp + g.u_rows - 1) / g.u_rows);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(tiles, sms));
    return fp16 ? launch_umma_a<__half>(f, Y, p, t, g, diag, s, grid, smem)
                : launch_umma_a<__nv_bfloat16>(f, Y, p, t, g, diag, s, grid, smem);
}

}  // namespace bfgc
