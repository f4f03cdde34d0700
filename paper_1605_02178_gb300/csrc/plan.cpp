// Host side of libbfgc: the FP64 coefficient fit (Sec. III), plan management and the
// C ABI entry points that validate arguments and enqueue the kernels.
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bfgc_adjoint.h"
#include "bfgc_internal.h"
#include "bfgc_recursive.h"
#include "bfgc_tc.h"

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

int window_radius(double sigma_s) { return (int)ceil(3.0 * sigma_s - 1e-9); }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Monomial coefficients of the Chebyshev polynomials, A[l][n] = coefficient of x^n in
// T_l, generated from T_{l+1} = 2 x T_l - T_{l-1} (eqs. (12), (13)).
std::vector<std::vector<double>> chebyshev_monomials(int N) {
    std::vector<std::vector<double>> A(N + 1, std::vector<double>(N + 2, 0.0));
    A[0][0] = 1.0;
    if (N >= 1) A[1][1] = 1.0;
    for (int l = 2; l <= N; ++l)
        for (int n = 0; n <= l; ++n)
            A[l][n] = (n > 0 ? 2.0 * A[l - 1][n - 1] : 0.0) - A[l - 2][n];
    return A;
}

// Coefficients of the polynomial in x/mu approximating exp(x) on [-mu, mu]:
// the Chebyshev interpolant at the zeros of T_{N+1} (eqs. (16), (18)) rewritten in
// monomials of x/mu (eq. (19) without its factor mu^-n).  Also the derivative of
// each coefficient with respect to mu.  T_l at the nodes is taken from eq. (11),
// T_l(cos t) = cos(l t).
void chebyshev_fit(int N, double mu, double* ct, double* dct_dmu) {
    const int M = N + 1;
    std::vector<double> d(M, 0.0), dd(M, 0.0);
    for (int k = 1; k <= M; ++k) {
        const double theta = kPi * (2.0 * k - 1.0) / (2.0 * M);
        const double xi = cos(theta);
        const double h = exp(mu * xi);
        for (int l = 0; l < M; ++l) {
            const double Tl = cos(l * theta);
            d[l] += h * Tl;
            dd[l] += xi * h * Tl;
        }
    }
    for (int l = 0; l < M; ++l) {
        const double w = (l == 0 ? 1.0 : 2.0) / M;
        d[l] *= w;
        dd[l] *= w;
    }
    auto A = chebyshev_monomials(N);
    for (int n = 0; n <= N; ++n) {
        double s = 0.0, ds = 0.0;
        for (int l = N; l >= n; --l) {
            s += d[l] * A[l][n];
            ds += dd[l] * A[l][n];
        }
        ct[n] = s;
        dct_dmu[n] = ds;
    }
}

void taylor_fit(int N, double mu, double* ct, double* dct_dmu) {
    // c_n = 1/n!, so c~_n = mu^n / n! and d c~_n / d mu = n mu^(n-1) / n!
    double fact = 1.0;
    for (int n = 0; n <= N; ++n) {
        if (n > 0) fact *= n;
        ct[n] = pow(mu, n) / fact;
        dct_dmu[n] = n > 0 ? n * pow(mu, n - 1) / fact : 0.0;
    }
}

void refit(bf_gc_plan_s* p) {
    p->t_c = 0.5 * (p->L + p->U);
    p->s_r = 0.5 * (p->U - p->L);
    p->mu = p->s_r * p->s_r / (p->sigma_r * p->sigma_r);
    double dct[BF_MAX_N + 1];
    if (p->poly == BF_POLY_TAYLOR)
        taylor_fit(p->N, p->mu, p->c_tilde, dct);
    else
        chebyshev_fit(p->N, p->mu, p->c_tilde, dct);
    p->kappa = 0.0;
    for (int n = 0; n <= p->N; ++n) {
        p->c[n] = p->c_tilde[n] * pow(p->mu, -(double)n);
        p->kappa = std::max(p->kappa, fabs(p->c_tilde[n]));
    }
    if (!(p->kappa > 0.0) || !isfinite(p->kappa)) p->kappa = 1.0;
    const double dmu_dsigma = -2.0 * p->mu / p->sigma_r;
    for (int n = 0; n <= p->N; ++n) p->dcoef_dsigma[n] = dct[n] * dmu_dsigma / p->kappa;

    // worst kernel error over a grid of intensities (t, tau) in [L, U]^2
    double err = 0.0;
    const int G = 129;
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b) {
            const double tau = p->L + (p->U - p->L) * a / (G - 1.0) - p->t_c;
            const double t = p->L + (p->U - p->L) * b / (G - 1.0) - p->t_c;
            const double x = (tau / p->s_r) * (t / p->s_r);
            double poly = 0.0;
            for (int n = p->N; n >= 0; --n) poly = poly * x + p->c_tilde[n];
            const double s2 = 2.0 * p->sigma_r * p->sigma_r;
            const double approx = exp(-tau * tau / s2) * exp(-t * t / s2) * poly;
            err = std::max(err, fabs(exp(-(t - tau) * (t - tau) / s2) - approx));
        }
    p->fit_err = isfinite(err) ? err : INFINITY;

    GcParams& g = p->gp;
    g.H = p->H; g.W = p->W; g.N = p->N; g.C = p->C; g.R = p->R;
    g.t_c = (float)p->t_c;
    g.inv_sr = (float)(1.0 / p->s_r);
    g.s_r = (float)p->s_r;
    g.half_mu = (float)(0.5 * p->mu);
    for (int n = 0; n < BF_MAX_C; ++n) g.coef[n] = n <= p->N ? (float)(p->c_tilde[n] / p->kappa) : 0.0f;
    // decisions on the FP32 sums unless bf_gc_forward hands the pixel to the FP64 refinement
    g.refine = nullptr;
    g.flag_rel = kFlagRelFp32;
    g.flag_abs = 0.0f;
    g.flag_abs_sum = 0.0f;
    g.flag_abs0 = 0.0f;
    g.clear_rel = (float)kIllcondRel;
    g.guard_rel = kGuardRel32;
    g.wait_ns = (unsigned long long)(p->wait_us * 1000.0);
    g.stall = p->stall;

    RefineParams& r = p->rp;
    r.H = p->H; r.W = p->W; r.N = p->N; r.C = p->C; r.R = p->R;
    r.t_c = p->t_c;
    r.inv_sr = 1.0 / p->s_r;
    r.s_r = p->s_r;
    r.half_mu = 0.5 * p->mu;
    for (int n = 0; n < BF_MAX_C; ++n) r.coef[n] = n <= p->N ? p->c_tilde[n] / p->kappa : 0.0;
    r.t_c32 = g.t_c;
    r.inv_sr32 = g.inv_sr;
    r.s_r32 = g.s_r;
    r.half_mu32 = g.half_mu;
    r.tier1_rel = kTier1Rel;
    for (int n = 0; n < BF_MAX_C; ++n) r.coef32[n] = g.coef[n];
    r.abs32 = kFlagAbsFp32;
    r.tier1 = 0;                                   // set per call from the storage precision
}

void make_taps(double sigma_s, int R, Taps* t, double* t64, float* t32) {
    double sum = 0.0;
    for (int d = -R; d <= R; ++d) sum += exp(-(double)d * d / (2.0 * sigma_s * sigma_s));
    t->R = R;
    for (int d = 0; d <= BF_MAX_R; ++d) {
        t64[d] = d <= R ? exp(-(double)d * d / (2.0 * sigma_s * sigma_s)) / sum : 0.0;
        t->g[d] = (float)t64[d];
        t32[d] = t->g[d];
    }
}

// The exact forms list pixels for the FP64 refinement (unless BF_OPT_REFINE = 0); the
// recursive form (an IIR stand-in for eq. (7), which a per-pixel window cannot reproduce)
// decides on its FP32 sums.
bool refines(const bf_gc_plan_s* p) { return p->form != BF_FORM_RECURSIVE && p->refine; }

// Bytes of the forward workspace before the refinement list (header included).
size_t fwd_body(const bf_gc_plan_s* p) {
    switch (p->form) {
    case BF_FORM_PLAIN:
        return BF_WS_HEADER + 2 * (size_t)p->C * bfgc::plain_plane_stride(p->H, p->W) * sizeof(float);
    case BF_FORM_FUSED:
        return BF_WS_HEADER + (size_t)p->C * bfgc::plain_plane_stride(p->H, p->W) * sizeof(float);
    case BF_FORM_FUSED_TC:
        return BF_WS_HEADER + round_up(bfgc::tc_workspace_bytes(bfgc::tc_geometry(p->H, p->W, p->R, p->C, p->tile_w), p->C), 256);
    case BF_FORM_RECURSIVE:
        return BF_WS_HEADER + 2 * (size_t)p->C * bfgc::plain_plane_stride(p->H, p->W) * sizeof(float) +
               (size_t)p->C * std::max(p->H, p->W) * p->R * sizeof(float);
    default:
        return 0;
    }
}

// Offset of the refinement list (one 32-bit pixel index per pixel at most) in the workspace.
size_t refine_list_offset(const bf_gc_plan_s* p) { return round_up(fwd_body(p), 256); }

size_t fwd_workspace(const bf_gc_plan_s* p) {
    if (!refines(p)) return fwd_body(p);
    return refine_list_offset(p) + round_up((size_t)p->H * p->W * sizeof(uint32_t), 256);
}

// Young and van Vliet (1995): scale q from sigma by their fit, b0..b3 cubic in q,
// B = 1 - (b1 + b2 + b3)/b0; the recursion uses a_k = b_k / b0.
bfgc::IirCoef iir_coefficients(double sigma, int P) {
    const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330 : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    const double q2 = q * q, q3 = q2 * q;
    const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    const double b2 = -(1.4281 * q2 + 1.26661 * q3);
    const double b3 = 0.422205 * q3;
    bfgc::IirCoef c;
    c.P = P;
    c.B = (float)(1.0 - (b1 + b2 + b3) / b0);
    c.a1 = (float)(b1 / b0);
    c.a2 = (float)(b2 / b0);
    c.a3 = (float)(b3 / b0);
    return c;
}

// Backward workspace (every form): header | X: C planes | Y: C planes | D: one plane |
// 2 * kAdjBlocks doubles.  Its prefix is the plain forward's workspace, so a plain forward
// with BF_OPT_SAVE_CHANNELS = 1 run on the same buffer leaves the filtered channels in X.
size_t bwd_workspace(const bf_gc_plan_s* p) {
    const size_t cs = bfgc::plain_plane_stride(p->H, p->W);
    return BF_WS_HEADER + (2 * (size_t)p->C + 1) * cs * sizeof(float) + 2 * bfgc::kAdjBlocks * sizeof(double);
}

// BF_FORM_AUTO: the tensor-core form with 16-bit storage while it exists (R <= 128), the fused
// FP32 form at FP32 while it costs at most twice the recursive form (measured), the recursive
// form beyond either
int auto_form(const bf_gc_plan_s* p) {
    if (p->precision != BF_PREC_FP32) return bfgc::tc_supported(p->R, p->C) ? BF_FORM_FUSED_TC : BF_FORM_RECURSIVE;
    return p->R <= BF_AUTO_FP32_EXACT_MAX_R && bfgc::fused_f32_supported(p->R) ? BF_FORM_FUSED : BF_FORM_RECURSIVE;
}

bool form_supported(const bf_gc_plan_s* p) {
    // the refinement list holds 32-bit pixel indices
    if (refines(p) && (unsigned long long)p->H * p->W > 0xFFFFFFFFull) return false;
    switch (p->form) {
    case BF_FORM_PLAIN:
        return p->precision == BF_PREC_FP32;
    case BF_FORM_FUSED:
        return p->precision == BF_PREC_FP32 && bfgc::fused_f32_supported(p->R);
    case BF_FORM_FUSED_TC:
        return (p->precision == BF_PREC_BF16 || p->precision == BF_PREC_FP16) && bfgc::tc_supported(p->R, p->C);
    case BF_FORM_RECURSIVE:
        // computed in FP32; chosen by BF_FORM_AUTO also when 16-bit storage was allowed
        return (p->precision == BF_PREC_FP32 || p->form_auto) && p->sigma_s >= 0.5;
    default:
        return false;
    }
}

// the last CUDA error a call of this thread turned into BF_ERR_CUDA (bf_last_cuda_error)
thread_local int g_last_cuda_error = 0;

bf_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return BF_OK;
    g_last_cuda_error = (int)e;
    return BF_ERR_CUDA;
}

// ---- optional event timing ---------------------------------------------------------
void prof_clear(Profiler& pr) {
    for (auto& m : pr.marks) cudaEventDestroy(m.ev);
    pr.marks.clear();
    pr.open = -1;
}

// Record the start of kernel `name` (and thereby the end of the previous one).  Every stage is
// also an NVTX range on the calling thread ("bfgc <stage>", host-side launch time), whether or
// not the event profiler is on; without an attached tool the NVTX calls return at once.
void prof_mark(bf_gc_plan_s* p, const char* name, cudaStream_t s) {
    Profiler& pr = p->prof;
    if (pr.nvtx_open) {
        nvtxRangePop();
        pr.nvtx_open = false;
    }
    if (name) {
        char label[64];
        std::snprintf(label, sizeof(label), "bfgc %s", name);
        nvtxRangePushA(label);
        pr.nvtx_open = true;
    }
    if (!pr.enabled) return;
    int k = -1;
    if (name) {
        for (size_t i = 0; i < pr.names.size(); ++i)
            if (pr.names[i] == name) k = (int)i;
        if (k < 0) {
            pr.names.push_back(name);
            pr.total_ms.push_back(0.0);
            pr.launches.push_back(0);
            k = (int)pr.names.size() - 1;
        }
    }
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return;
    cudaEventRecord(ev, s);
    pr.marks.push_back({k, ev});
    pr.open = k;
}

void prof_close(bf_gc_plan_s* p, cudaStream_t s) {
    if (p->prof.nvtx_open) {
        nvtxRangePop();
        p->prof.nvtx_open = false;
    }
    if (p->prof.enabled && p->prof.open >= 0) prof_mark(p, nullptr, s);
}

}  // namespace

extern "C" {

bf_status bf_gc_plan(int H, int W, double sigma_s, double sigma_r, int N, bf_gc_plan_t* out) {
    if (!out) return BF_ERR_INVALID_ARG;
    *out = nullptr;
    if (H < 1 || W < 1 || (long long)H * W > (1LL << 40) || !(sigma_s > 0.0) || !(sigma_r > 0.0) ||
        !isfinite(sigma_s) || !isfinite(sigma_r) || N < 1 || N > BF_MAX_N)
        return BF_ERR_INVALID_ARG;
    const int R = window_radius(sigma_s);
    if (R > BF_MAX_R) return BF_ERR_UNSUPPORTED;
    bf_gc_plan_s* p = new (std::nothrow) bf_gc_plan_s();
    if (!p) return BF_ERR_NOMEM;
    p->H = H; p->W = W; p->N = N; p->C = N + 2; p->R = R;
    p->sigma_s = sigma_s; p->sigma_r = sigma_r;
    p->L = 0.0; p->U = 255.0;
    p->form = BF_FORM_PLAIN; p->precision = BF_PREC_FP32; p->poly = BF_POLY_CHEBYSHEV; p->form_auto = false;
    p->save_channels = 0; p->tile_w = 0; p->refine = 1; p->used = false;
    p->wait_us = 1e6; p->stall = 0;
    refit(p);
    make_taps(sigma_s, R, &p->taps, p->rp.taps, p->rp.taps32);
    *out = p;
    return BF_OK;
}

bf_status bf_gc_plan_set(bf_gc_plan_t p, int option, double value) {
    if (!p || p->used || !isfinite(value)) return BF_ERR_INVALID_ARG;
    const int iv = (int)value;
    switch (option) {
    case BF_OPT_FORM:
        if (iv != value || iv < BF_FORM_PLAIN || iv > BF_FORM_FUSED) return BF_ERR_INVALID_ARG;
        p->form_auto = iv == BF_FORM_AUTO;
        p->form = p->form_auto ? auto_form(p) : iv;
        return BF_OK;
    case BF_OPT_PRECISION:
        if (iv != value || iv < BF_PREC_FP32 || iv > BF_PREC_FP16) return BF_ERR_INVALID_ARG;
        p->precision = iv;
        if (p->form_auto) p->form = auto_form(p);
        return BF_OK;
    case BF_OPT_RANGE_L:
    case BF_OPT_RANGE_U: {
        const double L = option == BF_OPT_RANGE_L ? value : p->L;
        const double U = option == BF_OPT_RANGE_U ? value : p->U;
        if (!(U > L)) return BF_ERR_INVALID_ARG;
        p->L = L;
        p->U = U;
        refit(p);
        return BF_OK;
    }
    case BF_OPT_POLY:
        if (iv != value || (iv != BF_POLY_CHEBYSHEV && iv != BF_POLY_TAYLOR)) return BF_ERR_INVALID_ARG;
        p->poly = iv;
        refit(p);
        return BF_OK;
    case BF_OPT_SAVE_CHANNELS:
        if (iv != value || (iv != 0 && iv != 1)) return BF_ERR_INVALID_ARG;
        p->save_channels = iv;
        return BF_OK;
    case BF_OPT_REFINE:
        if (iv != value || (iv != 0 && iv != 1)) return BF_ERR_INVALID_ARG;
        p->refine = iv;
        return BF_OK;
    case BF_OPT_WAIT_US:
        if (!(value >= 1.0 && value <= 1e7)) return BF_ERR_INVALID_ARG;
        p->wait_us = value;
        p->gp.wait_ns = (unsigned long long)(value * 1000.0);
        return BF_OK;
    case BF_OPT_STALL:
        if (iv != value || iv < 0 || iv > 2) return BF_ERR_INVALID_ARG;
        p->stall = iv;
        p->gp.stall = iv;
        return BF_OK;
    case BF_OPT_TILE_W:
        if (iv != value || (iv != 0 && iv != 64 && iv != 128 && iv != 256)) return BF_ERR_INVALID_ARG;
        if (iv > 64 && (p->R + 15) / 16 > 4) return BF_ERR_UNSUPPORTED;
        p->tile_w = iv;
        return BF_OK;
    default:
        return BF_ERR_INVALID_ARG;
    }
}

bf_status bf_gc_plan_info(bf_gc_plan_t p, bf_gc_info* o) {
    if (!p || !o) return BF_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->H = p->H; o->W = p->W; o->N = p->N; o->R = p->R; o->C = p->C;
    o->form = p->form; o->precision = p->precision; o->poly = p->poly;
    o->sigma_s = p->sigma_s; o->sigma_r = p->sigma_r; o->L = p->L; o->U = p->U;
    o->t_c = p->t_c; o->s_r = p->s_r; o->mu = p->mu; o->kappa = p->kappa; o->fit_err = p->fit_err;
    for (int n = 0; n <= p->N; ++n) {
        o->c[n] = p->c[n];
        o->c_tilde[n] = p->c_tilde[n];
    }
    return BF_OK;
}

bf_status bf_gc_workspace_size(bf_gc_plan_t p, size_t* fwd, size_t* bwd) {
    if (!p) return BF_ERR_INVALID_ARG;
    if (!form_supported(p)) return BF_ERR_UNSUPPORTED;
    if (fwd) *fwd = fwd_workspace(p);
    if (bwd) *bwd = bwd_workspace(p);
    return BF_OK;
}

bf_status bf_gc_forward(bf_gc_plan_t p, const float* f, float* out, void* ws, size_t ws_bytes,
                        bf_stream_t stream) {
    if (!p || !f || !out || !aligned(f, 16) || !aligned(out, 16)) return BF_ERR_INVALID_ARG;
    const size_t px = (size_t)p->H * p->W;
    if ((const char*)f < (const char*)(out + px) && (const char*)out < (const char*)(f + px))
        return BF_ERR_INVALID_ARG;
    if (!form_supported(p)) return BF_ERR_UNSUPPORTED;
    if (!ws || !aligned(ws, 256) || ws_bytes < fwd_workspace(p)) return BF_ERR_WORKSPACE;
    p->used = true;
    cudaStream_t s = (cudaStream_t)stream;
    DiagHeader* diag = (DiagHeader*)ws;
    cudaError_t e = cudaMemsetAsync(diag, 0, sizeof(DiagHeader), s);
    if (e != cudaSuccess) return BF_ERR_CUDA;
    char* body = (char*)ws + BF_WS_HEADER;
    // per-call parameters: the exact forms hand the pixels their FP32 sums cannot resolve to
    // the FP64 refinement, through the list at the end of this workspace
    GcParams gp = p->gp;
    if (refines(p)) {
        gp.refine = reinterpret_cast<uint32_t*>((char*)ws + refine_list_offset(p));
        gp.flag_rel = p->precision == BF_PREC_BF16   ? kFlagRelBf16
                      : p->precision == BF_PREC_FP16 ? kFlagRelFp16
                                                     : kFlagRelFp32;
        double a1 = 0.0;                                   // sum_n |coef_n|
        for (int n = 0; n <= p->N; ++n) a1 += fabs((double)gp.coef[n]);
        gp.flag_abs = p->precision == BF_PREC_FP16 ? kFlagAbsFp16 : kFlagAbsFp32;
        gp.flag_abs_sum = (float)(gp.flag_abs * a1);
        gp.flag_abs0 = gp.flag_abs * fabsf(gp.coef[0]);
        gp.clear_rel = gp.flag_rel;
    }
    switch (p->form) {
    case BF_FORM_PLAIN: {
        const size_t cs = bfgc::plain_plane_stride(p->H, p->W);
        float* X = (float*)body;
        float* Y = X + (size_t)p->C * cs;
        prof_mark(p, "build", s);
        if ((e = bfgc::launch_build(f, X, gp, cs, s)) != cudaSuccess) break;
        prof_mark(p, "hpass", s);
        if ((e = bfgc::launch_hpass(X, Y, gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
        prof_mark(p, "vpass", s);
        if ((e = bfgc::launch_vpass(Y, X, gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
        prof_mark(p, "combine", s);
        e = bfgc::launch_combine(f, X, out, gp, cs, diag, s);
        break;
    }
    case BF_FORM_FUSED: {
        const size_t cs = bfgc::plain_plane_stride(p->H, p->W);
        float* Y = (float*)body;
        prof_mark(p, "build_hpass_f32", s);
        if ((e = bfgc::launch_build_hpass_f32(f, Y, gp, p->taps, cs, s)) != cudaSuccess) break;
        prof_mark(p, "vpass_combine_f32", s);
        e = bfgc::launch_vpass_combine_f32(f, Y, out, gp, p->taps, cs, diag, s);
        break;
    }
    case BF_FORM_FUSED_TC: {
        const bfgc::TcGeom g = bfgc::tc_geometry(p->H, p->W, p->R, p->C, p->tile_w);
        const bool fp16 = p->precision == BF_PREC_FP16;
        prof_mark(p, "build_hpass_tc", s);
        // row pass: the Toeplitz operand in tensor memory (default), or in shared memory with
        // the tile width the plan asks for
        if ((e = p->tile_w ? bfgc::launch_build_hpass_umma(f, body, gp, p->taps, g, fp16, diag, s)
                           : bfgc::launch_build_hpass_tc(f, body, gp, p->taps, g, fp16, diag, s)) != cudaSuccess) break;
        prof_mark(p, "vpass_combine_tc", s);
        e = bfgc::launch_vpass_combine_tc(f, body, out, gp, p->taps, g, fp16, diag, s);
        break;
    }
    case BF_FORM_RECURSIVE: {
        const size_t cs = bfgc::plain_plane_stride(p->H, p->W);
        float* X = (float*)body;
        float* Y = X + (size_t)p->C * cs;
        float* tail = Y + (size_t)p->C * cs;
        const bfgc::IirCoef ic = iir_coefficients(p->sigma_s, p->R);
        prof_mark(p, "build", s);
        if ((e = bfgc::launch_build(f, X, gp, cs, s)) != cudaSuccess) break;
        prof_mark(p, "iir_rows", s);
        if ((e = bfgc::launch_iir(0, X, Y, tail, gp, ic, cs, p->C, s)) != cudaSuccess) break;   // result in X
        prof_mark(p, "iir_cols", s);
        if ((e = bfgc::launch_iir(1, X, Y, tail, gp, ic, cs, p->C, s)) != cudaSuccess) break;   // result in Y
        prof_mark(p, "combine", s);
        e = bfgc::launch_combine(f, Y, out, gp, cs, diag, s);
        break;
    }
    default:
        return BF_ERR_UNSUPPORTED;
    }
    if (e == cudaSuccess && refines(p)) {
        prof_mark(p, "refine_fp64", s);
        RefineParams rp = p->rp;
        rp.tier1 = p->precision != BF_PREC_FP32;
        e = bfgc::launch_refine(f, out, gp.refine, diag, rp, s);
    }
    prof_close(p, s);
    return cuda_status(e);
}

bf_status bf_gc_forward_host(bf_gc_plan_t p, const float* h_f, float* h_out, float* d_f,
                             float* d_out, void* ws, size_t ws_bytes, bf_stream_t stream) {
    if (!p || !h_f || !h_out || !d_f || !d_out) return BF_ERR_INVALID_ARG;
    const size_t bytes = (size_t)p->H * p->W * sizeof(float);
    cudaStream_t s = (cudaStream_t)stream;
    if (!form_supported(p)) return BF_ERR_UNSUPPORTED;
    if (!ws || !aligned(ws, 256) || ws_bytes < fwd_workspace(p)) return BF_ERR_WORKSPACE;
    if (cudaMemcpyAsync(d_f, h_f, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return BF_ERR_CUDA;
    bf_status st = bf_gc_forward(p, d_f, d_out, ws, ws_bytes, stream);
    if (st != BF_OK) return st;
    if (cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return BF_ERR_CUDA;
    return cuda_status(cudaStreamSynchronize(s));
}

bf_status bf_gc_backward(bf_gc_plan_t p, const float* f, const float* gout, float* gf,
                         double* gsigma, void* ws, size_t ws_bytes, bf_stream_t stream) {
    if (!p || !f || !gout || !gf || !aligned(f, 16) || !aligned(gout, 16) || !aligned(gf, 16) ||
        (gsigma && !aligned(gsigma, 8)))
        return BF_ERR_INVALID_ARG;
    if (!form_supported(p) || p->form == BF_FORM_RECURSIVE) return BF_ERR_UNSUPPORTED;
    if (!ws || !aligned(ws, 256) || ws_bytes < bwd_workspace(p)) return BF_ERR_WORKSPACE;
    p->used = true;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cs = bfgc::plain_plane_stride(p->H, p->W);
    float* X = (float*)((char*)ws + BF_WS_HEADER);
    float* Y = X + (size_t)p->C * cs;
    float* Dt = Y + (size_t)p->C * cs;
    double* partial = (double*)(Dt + cs);
    bfgc::AdjCoef ac{};
    for (int n = 0; n <= p->N; ++n) ac.dcoef[n] = (float)p->dcoef_dsigma[n];
    ac.inv_sigma3 = 1.0 / (p->sigma_r * p->sigma_r * p->sigma_r);
    cudaError_t e = cudaSuccess;
    do {
        if (!(p->save_channels && p->form == BF_FORM_PLAIN)) {      // filtered channels -> X
            if (bfgc::fused_f32_supported(p->R)) {
                // channels and row pass in one kernel (the plain form's operations, same bits)
                prof_mark(p, "build_hpass_f32", s);
                if ((e = bfgc::launch_build_hpass_f32(f, Y, p->gp, p->taps, cs, s)) != cudaSuccess) break;
            } else {
                prof_mark(p, "build", s);
                if ((e = bfgc::launch_build(f, X, p->gp, cs, s)) != cudaSuccess) break;
                prof_mark(p, "hpass", s);
                if ((e = bfgc::launch_hpass(X, Y, p->gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
            }
            prof_mark(p, "vpass", s);
            if ((e = bfgc::launch_vpass(Y, X, p->gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
        }
        prof_mark(p, "adjoint_lambda", s);
        if ((e = bfgc::launch_adjoint_lambda(f, gout, X, Y, Dt, partial, p->gp, ac, cs, s)) != cudaSuccess) break;
        prof_mark(p, "adjoint_vpass", s);       // K = V H, so K^T = H^T V^T
        if ((e = bfgc::launch_vpass_adjoint(Y, X, p->gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
        prof_mark(p, "adjoint_hpass", s);
        if ((e = bfgc::launch_hpass_adjoint(X, Y, p->gp, p->taps, cs, p->C, s)) != cudaSuccess) break;
        prof_mark(p, "adjoint_assemble", s);
        if ((e = bfgc::launch_adjoint_assemble(f, Y, Dt, gf, partial + bfgc::kAdjBlocks, p->gp, ac, cs, s)) !=
            cudaSuccess)
            break;
        if (gsigma) {
            prof_mark(p, "adjoint_reduce", s);
            e = bfgc::launch_adjoint_reduce(partial, 2 * bfgc::kAdjBlocks, gsigma, s);
        }
    } while (false);
    prof_close(p, s);
    return cuda_status(e);
}

bf_status bf_gc_diagnostics(bf_gc_plan_t p, const void* ws, bf_gc_diag* out, bf_stream_t stream) {
    if (!p || !ws || !out || !aligned(ws, 256)) return BF_ERR_INVALID_ARG;
    DiagHeader h;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return BF_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BF_ERR_CUDA;
    out->n_guarded = h.n_guarded;
    out->n_illcond = h.n_illcond;
    out->error_flags = h.error_flags;
    out->n_refined = h.n_flagged;
    out->n_refined_fp64 = h.n_refined64;
    return h.error_flags ? BF_ERR_TIMEOUT : BF_OK;
}

void bf_gc_plan_destroy(bf_gc_plan_t p) {
    if (!p) return;
    prof_clear(p->prof);
    delete p;
}

bf_status bf_gc_profile_enable(bf_gc_plan_t p, int enable) {
    if (!p) return BF_ERR_INVALID_ARG;
    prof_clear(p->prof);
    p->prof.names.clear();
    p->prof.total_ms.clear();
    p->prof.launches.clear();
    p->prof.enabled = enable != 0;
    return BF_OK;
}

bf_status bf_gc_profile_read(bf_gc_plan_t p, bf_kernel_time* out, int max_entries, int* n_entries) {
    if (!p || max_entries < 0 || (max_entries > 0 && !out)) return BF_ERR_INVALID_ARG;
    Profiler& pr = p->prof;
    if (!pr.marks.empty() && cudaEventSynchronize(pr.marks.back().ev) != cudaSuccess) return BF_ERR_CUDA;
    for (size_t i = 0; i + 1 < pr.marks.size(); ++i) {
        if (pr.marks[i].kernel < 0) continue;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, pr.marks[i].ev, pr.marks[i + 1].ev) != cudaSuccess) return BF_ERR_CUDA;
        pr.total_ms[pr.marks[i].kernel] += ms;
        pr.launches[pr.marks[i].kernel] += 1;
    }
    prof_clear(pr);
    const int n = (int)pr.names.size();
    for (int i = 0; i < n && i < max_entries; ++i) {
        memset(out[i].name, 0, sizeof(out[i].name));
        strncpy(out[i].name, pr.names[i].c_str(), sizeof(out[i].name) - 1);
        out[i].total_ms = pr.total_ms[i];
        out[i].launches = pr.launches[i];
    }
    if (n_entries) *n_entries = n;
    return BF_OK;
}

bf_status bf_direct(int H, int W, double sigma_s, double sigma_r, const float* f, float* out,
                    bf_stream_t stream) {
    if (H < 1 || W < 1 || !(sigma_s > 0.0) || !(sigma_r > 0.0) || !isfinite(sigma_s) ||
        !isfinite(sigma_r) || !f || !out || !aligned(f, 16) || !aligned(out, 16))
        return BF_ERR_INVALID_ARG;
    const int R = window_radius(sigma_s);
    if (R > BF_MAX_R) return BF_ERR_UNSUPPORTED;
    return cuda_status(bfgc::launch_direct(f, out, H, W, R, sigma_s, sigma_r, (cudaStream_t)stream));
}

bf_status bf_check_range(int H, int W, double L, double U, const float* f, unsigned long long* counts,
                         bf_stream_t stream) {
    if (H < 1 || W < 1 || !f || !counts || !isfinite(L) || !isfinite(U) || !(L <= U)) return BF_ERR_INVALID_ARG;
    return cuda_status(bfgc::launch_check_range(f, (size_t)H * W, (float)L, (float)U, counts, (cudaStream_t)stream));
}

const char* bf_status_string(bf_status s) {
    switch (s) {
    case BF_OK: return "ok";
    case BF_ERR_INVALID_ARG: return "invalid argument";
    case BF_ERR_UNSUPPORTED: return "unsupported";
    case BF_ERR_NOMEM: return "out of host memory";
    case BF_ERR_CUDA: return "CUDA error";
    case BF_ERR_TIMEOUT: return "device wait timed out";
    case BF_ERR_RANGE: return "input outside range";
    case BF_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    }
    return "unknown status";
}

const char* bf_version(void) { return "bfgc 0.1 (sm_103a)"; }

int bf_last_cuda_error(const char** name) {
    if (name) *name = g_last_cuda_error ? cudaGetErrorName((cudaError_t)g_last_cuda_error) : "cudaSuccess";
    return g_last_cuda_error;
}

}  // extern "C"
