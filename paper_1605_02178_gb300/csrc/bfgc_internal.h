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

// Diagnostics header at the start of a workspace.
struct DiagHeader {
    unsigned long long n_guarded;
    unsigned long long n_illcond;
    unsigned int error_flags;
    unsigned int pad[11];
};

// Per-plan scalars and coefficients, passed to kernels by value.
// u = (f - t_c) * inv_sr lies in [-1, 1] for f in [L, U];
// e = exp(-half_mu * u^2) = exp(-(f - t_c)^2 / (2 sigma_r^2));
// channel n holds e * u^n (F_n of eq. (6) rescaled by (sigma_r / s_r)^n), n = 0..C-1.
// coef[n] = c~_n / kappa with c~_n = mu^n c_n, so that
//   Q = sum_{n<=N} coef[n] u^n Fbar_n,  P = s_r sum_{n<=N} coef[n] u^n Fbar_{n+1}
// differ from eqs. (8)-(9) only by the common factor kappa (cancels in P/Q).
struct GcParams {
    int H, W, N, C, R;
    float t_c, inv_sr, s_r, half_mu;
    float coef[BF_MAX_C];
};

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
};

// Host-side plan.
struct bf_gc_plan_s {
    int H, W, N, R, C;
    double sigma_s, sigma_r, L, U;
    int form, precision, poly, save_channels, tile_w;
    bool form_auto;      // BF_FORM_AUTO was asked for: `form` is re-chosen on precision changes
    bool used;
    // derived (refit on option change)
    double t_c, s_r, mu, kappa, fit_err;
    double c[BF_MAX_N + 1], c_tilde[BF_MAX_N + 1];
    double dcoef_dsigma[BF_MAX_N + 1];  // d(c~_n)/d(sigma_r) / kappa
    GcParams gp;
    Taps taps;
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

// fused FP32 form: (build + row pass) -> C row-filtered planes of stride cs -> (column pass +
// ratio); false / cudaErrorInvalidValue where its shared-memory windows do not fit (large R)
bool fused_f32_supported(int R);
cudaError_t launch_build_hpass_f32(const float* f, float* Y, const GcParams& p, const Taps& t, size_t cs,
                                   cudaStream_t s);
cudaError_t launch_vpass_combine_f32(const float* f, const float* Y, float* out, const GcParams& p, const Taps& t,
                                     size_t cs, DiagHeader* diag, cudaStream_t s);

// exact filter of eq. (1)
cudaError_t launch_direct(const float* f, float* out, int H, int W, int R, double sigma_s,
                          double sigma_r, cudaStream_t s);

}  // namespace bfgc
