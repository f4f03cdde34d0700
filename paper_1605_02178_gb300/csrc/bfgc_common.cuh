// Device helpers shared by the kernels of libbfgc.
#pragma once

#include <algorithm>

#include "bfgc_internal.h"

namespace bfgc {

// Load of a run of L consecutive floats at element i of a 16-byte aligned array, whatever i's
// phase M = i mod 4: the elements before the first 16-byte boundary as a float and / or a
// float2, the aligned middle as float4s, the rest as a float2 and / or a float.  Nothing
// outside the run is read.  (M is a template argument so that every register index is static.)
template <int M, int L>
__device__ __forceinline__ void ldg_run_m(const float* __restrict__ p, float* v) {
    constexpr int HEAD = (4 - M) & 3;
    int j = 0;
    if (HEAD & 1) { v[0] = __ldg(p); j = 1; }
    if (HEAD >= 2) { const float2 t = __ldg(reinterpret_cast<const float2*>(p + j)); v[j] = t.x; v[j + 1] = t.y; j += 2; }
#pragma unroll
    for (int k = 0; k < (L - HEAD) / 4; ++k, j += 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p + j));
        v[j] = t.x; v[j + 1] = t.y; v[j + 2] = t.z; v[j + 3] = t.w;
    }
    if ((L - HEAD) % 4 >= 2) { const float2 t = __ldg(reinterpret_cast<const float2*>(p + j)); v[j] = t.x; v[j + 1] = t.y; j += 2; }
    if ((L - HEAD) % 2) v[j] = __ldg(p + j);
}
// v[0 .. L) = a[i .. i + L) for a 16-byte aligned array a
template <int L>
__device__ __forceinline__ void ldg_run(const float* __restrict__ a, size_t i, float* v) {
    switch ((unsigned)i & 3u) {
    case 0: ldg_run_m<0, L>(a + i, v); break;
    case 1: ldg_run_m<1, L>(a + i, v); break;
    case 2: ldg_run_m<2, L>(a + i, v); break;
    default: ldg_run_m<3, L>(a + i, v); break;
    }
}
// Half-sample symmetric extension of index p into [0, n) (period 2n).
__device__ __forceinline__ int mirror(int p, int n) {
    const int period = 2 * n;
    int q = p % period;
    if (q < 0) q += period;
    return q < n ? q : period - 1 - q;
}

// Decision of eq. (10) from the sums P, Q and Qa = sum |terms of Q| of a pixel at u: 0 = divide
// (conditioned), 1 = divide (ill-conditioned: |Q| < 1e-3 Qa, counted), 2 = guarded (output =
// input), 3 = hand the pixel to the FP64 refinement (p.refine set).  See GcParams for the two
// decision modes.  In refinement mode a pixel is also handed over when |Q| is within the
// absolute error that underflow of the stored channels can bring into Q: flag_abs (16 half
// spacings of the storage's smallest values) times A(|u|) = sum_n |coef_n| |u|^n, bounded by
// |coef_0| + |u| sum_n |coef_n| for |u| <= 1 and by sum_n |coef_n| |u|^N beyond.
__device__ __forceinline__ int ratio_decision(const GcParams& p, float u, float P, float Q, float Qa) {
    const bool bad = !(Qa > 0.0f) || !(Qa <= 3.0e38f) || !(fabsf(P) <= 3.0e38f);
    const float lhs = fabsf(Q);
    if (p.refine) {
        const float au = fabsf(u);
        const float bound = au <= 1.0f ? fmaf(au, p.flag_abs_sum, p.flag_abs * fabsf(p.coef[0]))
                                       : p.flag_abs_sum * __powf(au, (float)p.N);
        return (bad || !(lhs >= fmaf(p.flag_rel, Qa, bound))) ? 3 : 0;
    }
    if (bad || !(lhs >= p.guard_rel * Qa)) return 2;
    return lhs < (float)kIllcondRel * Qa ? 1 : 0;
}

// The common case of ratio_decision, cheaply: true only where ratio_decision is 0 (a finite,
// conditioned pixel in [L, U]); the rest take ratio_decision itself.
__device__ __forceinline__ bool ratio_clear(const GcParams& p, float u, float P, float Q, float Qa) {
    const float au = fabsf(u);
    return au <= 1.0f && Qa > 0.0f && Qa <= 3.0e38f && fabsf(P) <= 3.0e38f &&
           fabsf(Q) >= fmaf(p.clear_rel, Qa, fmaf(au, p.flag_abs_sum, p.flag_abs0));
}

// Per-pixel accumulation of eqs. (8)-(9) by Horner's rule in u = (f - t_c)/s_r over the
// filtered channels Z_m, visited from m = N+1 down to 0:
//   P = sum_{n=0}^{N} coef_n u^n Z_{n+1},  Q = sum_{n=0}^{N} coef_n u^n Z_n,
//   Qa = sum_{n=0}^{N} |coef_n u^n Z_n|  (scale of the terms of Q, for the guard).
struct RatioAcc {
    float u, au, P, Q, Qa;
    __device__ __forceinline__ void init(float u_) {
        u = u_;
        au = fabsf(u_);
        P = Q = Qa = 0.0f;
    }
    __device__ __forceinline__ void step(const GcParams& p, int m, float z) {
        if (m >= 1) P = fmaf(P, u, p.coef[m - 1] * z);
        if (m <= p.N) {
            const float q = p.coef[m] * z;
            Q = fmaf(Q, u, q);
            Qa = fmaf(Qa, au, fabsf(q));
        }
    }
    // Eq. (10): *how = ratio_decision(...); the input pixel is returned when the pixel is
    // guarded (2) or handed to the FP64 refinement (3, as a placeholder).  The FP32 division is
    // correctly rounded for the FP32 P and Q.
    __device__ __forceinline__ float finish(const GcParams& p, float f, int* how) const {
        *how = ratio_decision(p, u, P, Q, Qa);
        return *how >= 2 ? f : p.s_r * P / Q + p.t_c;
    }
};

// Append pixel i to the FP64 refinement list when `flag` is set.  Warp-aggregated: one
// atomic per group of converged lanes; safe in divergent code (each converged group takes
// its own slots).
__device__ __forceinline__ void refine_push(const GcParams& p, DiagHeader* diag, bool flag, uint32_t i) {
    const unsigned mask = __activemask();
    const unsigned b = __ballot_sync(mask, flag);
    if (!b) return;
    const int lane = (int)(threadIdx.x & 31), leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&diag->n_flagged, (unsigned long long)__popc(b));
    base = __shfl_sync(mask, base, leader);
    if (flag) p.refine[base + __popc(b & ((1u << lane) - 1u))] = i;
}

// Warp-aggregated update of the diagnostics counters.
__device__ __forceinline__ void count_diag(DiagHeader* diag, unsigned guarded, unsigned illcond) {
    const unsigned mask = __activemask();
    const unsigned g = __reduce_add_sync(mask, guarded);
    const unsigned d = __reduce_add_sync(mask, illcond);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(mask) - 1)) {
        if (g) atomicAdd(&diag->n_guarded, (unsigned long long)g);
        if (d) atomicAdd(&diag->n_illcond, (unsigned long long)d);
    }
}

}  // namespace bfgc
