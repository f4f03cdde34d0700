// Adjoint of the forward filter (the paper has no gradient; this is the exact derivative
// of the approximation computed by the FP32 forward).
//
// Forward, per pixel i (u = (f - t_c)/s_r, channels Fh_m = e u^m, Fbar_m = K Fh_m with K
// the separable mirror-extended Gaussian of eq. (7), coef_n = c~_n / kappa):
//   P = sum_n coef_n u^n Fbar_{n+1},  Q = sum_n coef_n u^n Fbar_n,  out = s_r P/Q + t_c.
// Given w = dL/dout:
//   Lambda_m = w s_r/Q (coef_{m-1} u^{m-1} [m >= 1] - (P/Q) coef_m u^m [m <= N])   (dL/dFbar_m)
//   D        = w s_r/Q (sum n coef_n u^{n-1} Fbar_{n+1} - (P/Q) sum n coef_n u^{n-1} Fbar_n)
//   M_m      = K^T Lambda_m   (K^T: same taps on zero-extended data, mirror images folded back;
//              k_plain.cu's row and column passes in adjoint mode)
//   dL/df    = (D + sum_m M_m (m Fh_{m-1} - mu u Fh_m)) / s_r       (de/du = -mu u e)
//   dL/dsigma_r = sum_i [ w s_r/Q sum_n coef'_n u^n (Fbar_{n+1} - (P/Q) Fbar_n) ]
//               + sum_j [ sum_m M_m Fh_m ] (f - t_c)^2 / sigma_r^3,
// coef'_n = d c~_n / d sigma_r / kappa (FP64 on the host; out is invariant to kappa).
// Guarded pixels (output = input) get Lambda = 0 and D = w s_r.
#include "bfgc_common.cuh"
#include "bfgc_adjoint.h"

namespace bfgc {

// ---------------------------------------------------------------------------------------
// Lambda channels, direct term D and the per-block sums of the coefficient term.
__global__ void __launch_bounds__(256) k_adjoint_lambda(const float* __restrict__ f, const float* __restrict__ gout,
                                                        const float* __restrict__ Z, float* __restrict__ Lam,
                                                        float* __restrict__ Dterm, double* __restrict__ partial,
                                                        const GcParams p, const AdjCoef ac, size_t cs, size_t px) {
    double local = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < px; i += stride) {
        const float fv = f[i], w = gout[i];
        const float u = (fv - p.t_c) * p.inv_sr;
        RatioAcc acc;
        acc.init(u);
        // Horner for P, Q plus the u-derivative sums and the coefficient-derivative sums
        float dP = 0.0f, dQ = 0.0f, sP = 0.0f, sQ = 0.0f;
        for (int m = p.C - 1; m >= 0; --m) {
            const float z = Z[(size_t)m * cs + i];
            // d/du of Horner: (acc)' = acc' u + acc
            if (m >= 1) {
                dP = fmaf(dP, u, acc.P);
                sP = fmaf(sP, u, ac.dcoef[m - 1] * z);
            }
            if (m <= p.N) {
                dQ = fmaf(dQ, u, acc.Q);
                sQ = fmaf(sQ, u, ac.dcoef[m] * z);
            }
            acc.step(p, m, z);
        }
        int how;
        acc.finish(p, fv, &how);
        if (how == 2) {
            for (int m = 0; m < p.C; ++m) Lam[(size_t)m * cs + i] = 0.0f;
            Dterm[i] = w * p.s_r;
            continue;
        }
        const float B = acc.P / acc.Q;
        const float k = w * p.s_r / acc.Q;
        // Lambda_m for m = 0..C-1 with u^m built upward
        float um1 = 0.0f, um = 1.0f;          // u^(m-1), u^m
        for (int m = 0; m < p.C; ++m) {
            float l = 0.0f;
            if (m >= 1) l = p.coef[m - 1] * um1;
            if (m <= p.N) l = fmaf(-B * p.coef[m], um, l);
            Lam[(size_t)m * cs + i] = k * l;
            um1 = um;
            um *= u;
        }
        Dterm[i] = k * (dP - B * dQ);
        local += (double)(k * (sP - B * sQ));
    }
    // block sum (fixed order per block -> deterministic)
    __shared__ double red[256];
    red[threadIdx.x] = local;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------------------
// dL/df and the per-block sums of the e-term of dL/dsigma_r.
__global__ void __launch_bounds__(256) k_adjoint_assemble(const float* __restrict__ f, const float* __restrict__ Mch,
                                                          const float* __restrict__ Dterm, float* __restrict__ gf,
                                                          double* __restrict__ partial, const GcParams p,
                                                          const AdjCoef ac, size_t cs, size_t px) {
    double local = 0.0;
    const float mu = 2.0f * p.half_mu;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < px; i += stride) {
        const float fv = f[i];
        const float u = (fv - p.t_c) * p.inv_sr;
        const float e = expf(-p.half_mu * u * u);
        float gu = Dterm[i], se = 0.0f;
        float fm1 = 0.0f, fm = e;                      // Fh_{m-1}, Fh_m
        for (int m = 0; m < p.C; ++m) {
            const float mm = Mch[(size_t)m * cs + i];
            gu = fmaf(mm, fmaf((float)m, fm1, -mu * u * fm), gu);
            se = fmaf(mm, fm, se);
            fm1 = fm;
            fm *= u;
        }
        gf[i] = gu * p.inv_sr;
        const double g = (double)fv - (double)p.t_c;
        local += (double)se * g * g * ac.inv_sigma3;
    }
    __shared__ double red[256];
    red[threadIdx.x] = local;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Sum of the block partials in a fixed order.
__global__ void k_adjoint_reduce(const double* __restrict__ partial, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------------------
cudaError_t launch_adjoint_lambda(const float* f, const float* gout, const float* Z, float* Lam, float* Dterm,
                                  double* partial, const GcParams& p, const AdjCoef& ac, size_t cs, cudaStream_t s) {
    const size_t px = (size_t)p.H * p.W;
    k_adjoint_lambda<<<kAdjBlocks, 256, 0, s>>>(f, gout, Z, Lam, Dterm, partial, p, ac, cs, px);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_assemble(const float* f, const float* Mch, const float* Dterm, float* gf, double* partial,
                                    const GcParams& p, const AdjCoef& ac, size_t cs, cudaStream_t s) {
    const size_t px = (size_t)p.H * p.W;
    k_adjoint_assemble<<<kAdjBlocks, 256, 0, s>>>(f, Mch, Dterm, gf, partial, p, ac, cs, px);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(const double* partial, int n, double* out, cudaStream_t s) {
    k_adjoint_reduce<<<1, 256, 0, s>>>(partial, n, out);
    return cudaGetLastError();
}

}  // namespace bfgc
