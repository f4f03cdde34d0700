// Internal declarations shared by the host plan and the CUDA kernels of libbfgc.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bfgc.h"

#define BF_MAX_C 64          // channels n = 0..N+1, N <= BF_MAX_N
#define BF_MAX_R 255         // largest window half-width accepted by the direct forms
#define BF_TC_MAX_A 8        // tensor-core forms: R <= 16 * BF_TC_MAX_A
#define BF_WS_HEADER 256     // bytes at the start of every workspace (diagnostics)

// Diagnostics header at the start of a workspace.  n_flagged is also the length of the
// FP64 refinement list of the exact forms (see GcParams::refine).
struct DiagHeader {
    unsigned long long n_guarded;
    unsigned long long n_illcond;
    unsigned int error_flags;
    unsigned int pad0;
    unsigned long long n_flagged;
    unsigned long long n_refined64;    // listed pixels that went on to the FP64 tier
    unsigned int pad[6];
};

// Per-plan scalars and coefficients, passed to kernels by value.
// u = (f - t_c) * inv_sr lies in [-1, 1] for f in [L, U];
// e = exp(-half_mu * u^2) = exp(-(f - t_c)^2 / (2 sigma_r^2));
// channel n holds e * u^n (F_n of eq. (6) rescaled by (sigma_r / s_r)^n), n = 0..C-1.
// coef[n] = c~_n / kappa with c~_n = mu^n c_n, so that
//   Q = sum_{n<=N} coef[n] u^n Fbar_n,  P = s_r sum_{n<=N} coef[n] u^n Fbar_{n+1}
// differ from eqs. (8)-(9) only by the common factor kappa (cancels in P/Q).
//
// Division of eq. (10).  With `refine` set (the exact forms), a pixel whose FP32 sums give
// |Q| < flag_rel * Qa (Qa = sum |terms of Q|), or no positive finite Qa, is not divided here:
// its index is appended to the list `refine` (length in DiagHeader::n_flagged) and the pixel
// is recomputed from f in FP64 by k_refine_fp64, which takes the guard decision and the
// division in FP64.  flag_rel is at least 1e-3 and covers the storage precision's error in Q.
// The test also refines pixels whose |Q| is within flag_abs sum_n |coef_n| |u|^n of zero (the
// error that underflow of the stored channels can bring; flag_abs_sum = flag_abs sum_n |coef_n|),
// see ratio_decision.
// Without `refine` (the recursive form, and the adjoint), the decision is taken on the FP32
// sums: output = input when |Q| < guard_rel * Qa or Qa is not positive and finite.
struct GcParams {
    int H, W, N, C, R;
    float t_c, inv_sr, s_r, half_mu;
    float flag_rel, flag_abs, flag_abs_sum, guard_rel;
    // ratio_clear: ratio_decision is 0 (divide, nothing to count) when |u| <= 1, the sums are
    // finite and |Q| >= clear_rel Qa + flag_abs0 + |u| flag_abs_sum (clear_rel = flag_rel with the
    // refinement, 1e-3 without; flag_abs0 = flag_abs |coef_0|)
    float clear_rel, flag_abs0;
    uint32_t* refine;
    // bound of one pipeline wait in the tensor-core kernels (BF_OPT_WAIT_US), and the test-only
    // stall of BF_OPT_STALL (0: none; 1: the row pass's first build group withholds its first
    // tile; 2: the column pass's TMA producer withholds its first stage)
    unsigned long long wait_ns;
    int stall;
    float coef[BF_MAX_C];
};

// The plan for the refinement kernel (k_refine.cu), in FP64 and FP32: u = (f - t_c) inv_sr,
// channels exp(-half_mu u^2) u^n, coef[n] = c~_n / kappa, taps[d] = normalised g(d), d = 0..R.
// tier1: the form stores 16-bit channels, so a listed pixel is first recomputed in FP32 and
// accepted there when |Q| >= tier1_rel Qa + abs32 sum_n |coef_n| |u|^n.
struct RefineParams {
    int H, W, N, C, R;
    int tier1;
    double t_c, inv_sr, s_r, half_mu;
    double coef[BF_MAX_C];
    double taps[BF_MAX_R + 1];
    float t_c32, inv_sr32, s_r32, half_mu32, tier1_rel, abs32;
    float coef32[BF_MAX_C];
    float taps32[BF_MAX_R + 1];
};
constexpr float kTier1Rel = 1e-2f;

// Relative guard of eq. (10) in FP64 (the oracle's delta) and the ill-conditioning mark.
constexpr double kGuardRel64 = 1e-12;
constexpr double kIllcondRel = 1e-3;
// Refinement thresholds flag_rel by channel storage: FP32 (1e-3, the ill-conditioning mark);
// BF16 and FP16, where the stored channels carry relative errors of up to a few times 2^-9
// and 2^-11 (the stored row-pass output, and the 16-bit channels and taps of the banded
// products), which reach Q at that size relative to the sum of its terms: 1/16 and 1/128, an
// eightfold margin over four units of storage rounding.
constexpr float kFlagRelFp32 = 1e-3f;
constexpr float kFlagRelBf16 = 0.0625f;
constexpr float kFlagRelFp16 = 0.0078125f;
// Absolute part of the refinement test, per unit of sum_n |coef_n| |u|^n (see ratio_decision):
// FP32 and BF16 channels lose relative precision below the smallest normal value 2^-126, so a
// Q within 2^-123 is refined; FP16 channels (stored times 2^14, the units in which the sums are
// taken) round with an absolute error of up to 2^-25 near zero, and a Q within 16 such errors
// (2^-21) is refined.
constexpr float kFlagAbsFp32 = 9.4039548065783e-38f;   // 2^-123
constexpr float kFlagAbsFp16 = 4.76837158203125e-7f;   // 2^-21
// Guard threshold where the decision is taken on FP32 sums: below 2^-17 Qa, Q is at the
// level of the rounding error of the FP32 sums of about N terms.
constexpr float kGuardRel32 = 7.62939453125e-6f;

// Normalised 1-D spatial taps g[|d|], d = -R..R, sum over d equal to one.
// (The paper's unnormalised g_s of Sec. I; the scale cancels in P/Q.)
struct Taps {
    int R;
    float g[BF_MAX_R + 1];
};

// Optional per-kernel event timing of a plan's launches.
struct Profiler {
    bool enabled = false;
    struct Mark {
        int kernel;              // index into names, or -1 for the closing event
        cudaEvent_t ev;
    };
    std::vector<Mark> marks;     // in recording order, per stream sequence
    std::vector<std::string> names;
    std::vector<double> total_ms;
    std::vector<unsigned long long> launches;
    int open = -1;               // kernel whose start mark is the last one recorded
    bool nvtx_open = false;      // an NVTX stage range is open on the calling thread
};

// Host-side plan.
struct bf_gc_plan_s {
    int H, W, N, R, C;
    double sigma_s, sigma_r, L, U;
    int form, precision, poly, save_channels, tile_w;
    int refine;          // BF_OPT_REFINE: FP64 refinement in the exact forms (default 1)
    double wait_us;      // BF_OPT_WAIT_US
    int stall;           // BF_OPT_STALL (testing the bounded waits)
    bool form_auto;      // BF_FORM_AUTO was asked for: `form` is re-chosen on precision changes
    bool used;
    // derived (refit on option change)
    double t_c, s_r, mu, kappa, fit_err;
    double c[BF_MAX_N + 1], c_tilde[BF_MAX_N + 1];
    double dcoef_dsigma[BF_MAX_N + 1];  // d(c~_n)/d(sigma_r) / kappa
    GcParams gp;
    Taps taps;
    RefineParams rp;     // FP64 plan of the refinement kernel
    Profiler prof;
};

// ---- launchers (return cudaGetLastError() after enqueueing) --------------------------
namespace bfgc {

// plain form: channel planes of stride cs floats
size_t plain_plane_stride(int H, int W);
cudaError_t launch_build(const float* f, float* X, const GcParams& p, size_t cs, cudaStream_t s);
cudaError_t launch_hpass(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                         int planes, cudaStream_t s);
cudaError_t launch_vpass(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                         int planes, cudaStream_t s);
cudaError_t launch_combine(const float* f, const float* Z, float* out, const GcParams& p,
                           size_t cs, DiagHeader* diag, cudaStream_t s);
// adjoints of the row and column passes (zero extension, mirror images folded back)
cudaError_t launch_hpass_adjoint(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                 int planes, cudaStream_t s);
cudaError_t launch_vpass_adjoint(const float* X, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                 int planes, cudaStream_t s);

// fused FP32 form: (build + row pass) -> C row-filtered planes of stride cs -> (column pass +
// ratio); false / cudaErrorInvalidValue where its shared-memory windows do not fit (large R)
bool fused_f32_supported(int R);
cudaError_t launch_build_hpass_f32(const float* f, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                   cudaStream_t s);
cudaError_t launch_vpass_combine_f32(const float* f, const float* Y, float* out, const GcParams& p, const Taps& t,
                                     size_t cs, DiagHeader* diag, cudaStream_t s);

// FP64 recomputation of the listed pixels (k_refine.cu)
// counts[0] = pixels of f[0 .. n) outside [L, U] (finite), counts[1] = non-finite ones
cudaError_t launch_check_range(const float* f, size_t n, float L, float U, unsigned long long* counts, cudaStream_t s);
cudaError_t launch_refine(const float* f, float* out, const uint32_t* list, DiagHeader* diag,
                          const RefineParams& rp, cudaStream_t s);

// exact filter of eq. (1)
cudaError_t launch_direct(const float* f, float* out, int H, int W, int R, double sigma_s,
                          double sigma_r, cudaStream_t s);

}  // namespace bfgc
