// Device helpers of the tensor-core kernels (k_rows_tc.cu, k_umma.cu, k_tc.cu): shared-memory
// addresses, bounded mbarrier waits, tensor-memory loads and stores, 16-bit packing.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "bfgc_internal.h"

namespace bfgc {
namespace tc {

constexpr unsigned kWaitNs = 1000000000u;        // bound of a drain wait, and the default bound of
                                                 // a pipeline wait (GcParams::wait_ns)
// Taps staged in shared memory for the Toeplitz fills: the lanes of a warp read different taps,
// and reading them from the kernel-parameter bank serialises (one access per distinct address)
constexpr int kTapsSmem = 132;                   // >= R + 1 for R <= 128 (ceil(R/16) <= 8)
constexpr unsigned kSuspendNs = 20000u;          // suspend-time hint of one try_wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" :: "r"(su32(bar)), "r"(bytes)
                 : "memory");
}
// try_wait with a suspend-time hint: a waiting warp sleeps until the phase completes (or the
// hint runs out) instead of spinning and taking issue slots from the working warps
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(bar)), "r"(parity), "r"(kSuspendNs) : "memory");
    return ok != 0;
}
// try_wait without a suspend hint (returns at once): for waits on the critical path, where a
// sleeping warp would add its wake-up latency to every hand-off
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` of `bar` (every waiter walks its barrier's phases in
// order, so the phase before the awaited one is complete).  Gives up when another role raised
// the abort flag, or (raising it, and or-ing `flag` into the workspace's error flags) after
// `limit_ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                                DiagHeader* diag, unsigned flag, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit_ns) break;
    }
    *abort_flag = 1;
    atomicOr(&diag->error_flags, flag);
    return false;
}
// As mbar_wait_abort, polling without the suspend hint
__device__ __forceinline__ bool mbar_wait_abort_poll(uint64_t* bar, unsigned parity, volatile int* abort_flag,
                                                     DiagHeader* diag, unsigned flag, uint64_t limit_ns) {
    if (mbar_poll(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (unsigned i = 0;; ++i) {
        if (mbar_poll(bar, parity)) return true;
        if ((i & 15) == 15) {
            if (*abort_flag) return false;
            if (global_ns() - t0 > limit_ns) break;
        }
    }
    *abort_flag = 1;
    atomicOr(&diag->error_flags, flag);
    return false;
}
// Bounded wait without abort (draining asynchronous work before the CTA exits); false if the
// bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

// Shared-memory matrix descriptor with the 128-byte swizzle: start address, leading and stride
// byte offsets (>> 4), descriptor version 1 (bit 46), swizzle mode 2 (bits 61..63).  K-major
// operands: 8-row groups 1024 bytes apart (SBO), LBO unused (16).  MN-major operands with 64
// elements per line: 8-line (K) groups 1024 bytes apart, 64-element MN blocks `lbo` apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr, uint32_t lbo = 16) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// FP16 channels are stored times 2^14: |e u^n| <= 1, so the scaled channels and their
// Gaussian averages stay below 2^14 (FP16 max 65504), while the high powers of mid-range
// pixels move out of the FP16 subnormal range.  A power of two is exact, and a common
// factor of every channel cancels in P/Q and in the relative division guard.
template <typename T> struct ChannelScale { static constexpr float value = 1.0f; };
template <> struct ChannelScale<__half> { static constexpr float value = 16384.0f; };

template <typename T> __device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <> __device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <typename T> __device__ __forceinline__ uint16_t one16(float v);
template <> __device__ __forceinline__ uint16_t one16<__nv_bfloat16>(float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}
template <> __device__ __forceinline__ uint16_t one16<__half>(float v) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    // load and wait in one statement: the registers are defined only once the wait is done
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* z) {
    uint32_t v[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) z[j] = __uint_as_float(v[j]);
}
// Split-phase load of 8 consecutive 32-bit columns of this warp's 32 lanes: tmem_ld8_start
// issues it, tmem_wait8 waits for every load of the thread issued so far.  The registers pass
// through the wait (in-out operands), so no use of them can be scheduled before it; between the
// two the thread can compute on registers of an earlier load.
__device__ __forceinline__ void tmem_ld8_start(uint32_t taddr, uint32_t* v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_wait8(uint32_t* v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                 :: "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// Two FP32 lanes in one 64-bit register (packed f32x2 arithmetic: one instruction for two
// products or two multiply-adds)
__device__ __forceinline__ uint64_t f2_make(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(uint64_t a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ uint64_t f2_abs(uint64_t a) { return a & 0x7FFFFFFF7FFFFFFFull; }

}  // namespace tc
}  // namespace bfgc
