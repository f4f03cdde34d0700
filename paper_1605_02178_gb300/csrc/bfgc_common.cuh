// Device helpers shared by the kernels of libbfgc.
#pragma once

#include <algorithm>

#include "bfgc_internal.h"

namespace bfgc {

// Half-sample symmetric extension of index p into [0, n) (period 2n).
__device__ __forceinline__ int mirror(int p, int n) {
    const int period = 2 * n;
    int q = p % period;
    if (q < 0) q += period;
    return q < n ? q : period - 1 - q;
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
    // Eq. (10) with the division guard; *how: 0 = conditioned, 1 = ill-conditioned
    // (|Q| < 1e-3 Qa, counted), 2 = guarded (|Q| < 1e-12 Qa, non-finite, or all terms zero):
    // the input pixel is returned.  The division is FP32 in every case: P and Q are FP32
    // values, so their FP32 quotient is already correctly rounded.
    __device__ __forceinline__ float finish(const GcParams& p, float f, int* how) const {
        if (!(fabsf(Q) >= 1e-12f * Qa) || !(Qa > 0.0f)) {
            *how = 2;
            return f;
        }
        *how = fabsf(Q) < 1e-3f * Qa ? 1 : 0;
        return p.s_r * P / Q + p.t_c;
    }
};

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
