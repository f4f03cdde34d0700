// Recomputation of the pixels whose denominator the forms' stored channels cannot resolve: the
// division of eq. (10) where Q is small against the sum of its terms.
//
// The exact forms list such pixels (GcParams::refine).  For each listed pixel i this kernel
// evaluates, from the input image alone,
//   Fbar_n(i) = sum_{|dy|,|dx| <= R} g(dy) g(dx) e(j) u(j)^n,  j = i + (dy, dx) mirrored
//               (eq. (7) of the channels of eq. (6) after the centring of eq. (17), in the
//               rescaled variable u = (f - t_c)/s_r, e = exp(-(f - t_c)^2 / (2 sigma_r^2))),
//   Q = sum_{n<=N} coef_n u^n Fbar_n,  P = s_r sum_{n<=N} coef_n u^n Fbar_{n+1}   (eqs. (8), (9)),
//   Qa = sum_{n<=N} |coef_n u^n Fbar_n|,
// in two tiers.  Tier 1 (forms with 16-bit channels, whose trouble is storage precision):
// the sums in FP32 from the input; if |Q| >= 1e-2 Qa (plus the underflow allowance, as in
// ratio_decision) the pixel is divided in FP32 and done.  Tier 2 (every other listed pixel,
// and every listed pixel of the FP32 forms): the sums in FP64 and the guard of eq. (10) in
// FP64: the output is the input pixel when |Q| < 1e-12 Qa or Qa is not positive (counted as
// guarded), else P/Q + t_c divided in FP64 (counted as ill-conditioned when |Q| < 1e-3 Qa).
// One warp per listed pixel: the lanes split the columns of each window row, each lane
// accumulates its share of every channel, and a warp reduction gives the sums.  Work is
// proportional to the list's length, which is zero wherever the range-kernel fit converges
// on images without isolated high-contrast pixels.
#include "bfgc_common.cuh"

namespace bfgc {

namespace {

constexpr int kRefWarps = 8;                       // warps per block

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int mirror_fast(int p, int n) { return (unsigned)p < (unsigned)n ? p : mirror(p, n); }

__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }

// P, Q, Qa of the pixel (y, x) with every step in type T (FP32 or FP64); CH channels per walk
// over the window.  taps / coef / scalars in T.
template <typename T, int CH>
__device__ __forceinline__ void window_sums(const float* __restrict__ f, const RefineParams& rp, const T* taps,
                                            const T* coef, T t_c, T inv_sr, T half_mu, int y, int x, T u0, int lane,
                                            T& P, T& Q, T& Qa) {
    P = Q = Qa = T(0);
    T um = T(1), um1 = T(0);                           // u0^m and u0^(m-1) for the channel m in hand
    for (int n0 = 0; n0 < rp.C; n0 += CH) {
        T Fb[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) Fb[k] = T(0);
        for (int dy = -rp.R; dy <= rp.R; ++dy) {
            const T wy = taps[dy < 0 ? -dy : dy];
            const float* row = f + (size_t)mirror_fast(y + dy, rp.H) * rp.W;
            for (int dx = lane - rp.R; dx <= rp.R; dx += 32) {
                const T uj = ((T)__ldg(row + mirror_fast(x + dx, rp.W)) - t_c) * inv_sr;
                T pw = wy * taps[dx < 0 ? -dx : dx] * exp_t(-half_mu * uj * uj);
                for (int k = 0; k < n0; ++k) pw *= uj;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    Fb[k] += pw;
                    pw *= uj;
                }
            }
        }
        // channel m = n0 + k enters Q with coef_m u0^m (m <= N) and P with coef_{m-1} u0^(m-1)
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const T s = warp_sum(Fb[k]);
            const int m = n0 + k;
            if (m < rp.C) {
                if (m <= rp.N) {
                    const T q = coef[m] * um * s;
                    Q += q;
                    Qa += q < T(0) ? -q : q;
                }
                if (m >= 1) P += coef[m - 1] * um1 * s;
                um1 = um;
                um *= u0;
            }
        }
    }
}

}  // namespace

// CH: channels accumulated per walk over the window (CH >= min(C, 32); C > 32 takes two walks).
template <int CH>
__global__ void __launch_bounds__(32 * kRefWarps) k_refine(const float* __restrict__ f, float* __restrict__ out,
                                                           const uint32_t* __restrict__ list, DiagHeader* diag,
                                                           const RefineParams rp) {
    // the list was written by the previous kernel on the stream (programmatic dependent launch:
    // wait here until it has completed and its writes are visible)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const unsigned long long px = (unsigned long long)rp.H * rp.W;
    unsigned long long count = *reinterpret_cast<volatile unsigned long long*>(&diag->n_flagged);
    count = count < px ? count : px;
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * kRefWarps;
    unsigned guarded = 0, illcond = 0, fp64 = 0;
    for (unsigned long long e = (unsigned long long)blockIdx.x * kRefWarps + (threadIdx.x >> 5); e < count;
         e += nwarps) {
        const uint32_t i = list[e];
        const int y = (int)(i / (uint32_t)rp.W), x = (int)(i - (uint32_t)y * (uint32_t)rp.W);
        if (rp.tier1) {
            const float u0 = (f[i] - rp.t_c32) * rp.inv_sr32;
            float P, Q, Qa;
            window_sums<float, CH>(f, rp, rp.taps32, rp.coef32, rp.t_c32, rp.inv_sr32, rp.half_mu32, y, x, u0, lane,
                                   P, Q, Qa);
            // the underflow allowance of ratio_decision, with A(|u|) = sum_n |coef_n| |u|^n
            float A = 0.0f;
            for (int n = rp.N; n >= 0; --n) A = fmaf(A, fabsf(u0), fabsf(rp.coef32[n]));
            const float tabs = rp.abs32 * A;
            if (Qa > 0.0f && Qa <= 3.0e38f && fabsf(P) <= 3.0e38f && fabsf(Q) >= fmaf(rp.tier1_rel, Qa, tabs)) {
                if (lane == 0) out[i] = rp.s_r32 * P / Q + rp.t_c32;
                continue;
            }
        }
        const double u0 = ((double)f[i] - rp.t_c) * rp.inv_sr;
        double P, Q, Qa;
        window_sums<double, CH>(f, rp, rp.taps, rp.coef, rp.t_c, rp.inv_sr, rp.half_mu, y, x, u0, lane, P, Q, Qa);
        if (lane == 0) {
            ++fp64;
            if (!(fabs(Q) >= kGuardRel64 * Qa) || !(Qa > 0.0)) {
                out[i] = f[i];
                ++guarded;
            } else {
                out[i] = (float)(rp.s_r * P / Q + rp.t_c);
                illcond += fabs(Q) < kIllcondRel * Qa;
            }
        }
    }
    if (lane == 0) {
        if (guarded) atomicAdd(&diag->n_guarded, (unsigned long long)guarded);
        if (illcond) atomicAdd(&diag->n_illcond, (unsigned long long)illcond);
        if (fp64) atomicAdd(&diag->n_refined64, (unsigned long long)fp64);
    }
}

namespace {

template <int CH>
cudaError_t launch_refine_ch(const float* f, float* out, const uint32_t* list, DiagHeader* diag,
                             const RefineParams& rp, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long px = (unsigned long long)rp.H * rp.W;
    const unsigned long long want = (px + kRefWarps - 1) / kRefWarps;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>(want, 2ull * sms)));
    cfg.blockDim = dim3(32 * kRefWarps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    // programmatic dependent launch: the launch overlaps the end of the previous kernel, whose
    // completion the kernel awaits (griddepcontrol.wait) before it reads the list
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_refine<CH>, f, out, list, diag, rp);
}

}  // namespace

cudaError_t launch_refine(const float* f, float* out, const uint32_t* list, DiagHeader* diag, const RefineParams& rp,
                          cudaStream_t s) {
    const int c = std::min(rp.C, 32);
    cudaError_t e;
    if (c <= 8) e = launch_refine_ch<8>(f, out, list, diag, rp, s);
    else if (c <= 16) e = launch_refine_ch<16>(f, out, list, diag, rp, s);
    else if (c <= 24) e = launch_refine_ch<24>(f, out, list, diag, rp, s);
    else e = launch_refine_ch<32>(f, out, list, diag, rp, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace bfgc
