// Launchers of the adjoint (backward) kernels, k_adjoint.cu.
#pragma once

#include "bfgc_internal.h"

namespace bfgc {

constexpr int kAdjBlocks = 152 * 8;   // grid of the per-pixel adjoint kernels (block partials)

// Coefficient derivatives for dL/dsigma_r.
struct AdjCoef {
    float dcoef[BF_MAX_C];   // d(c~_n)/d(sigma_r) / kappa, n = 0..N
    double inv_sigma3;       // 1 / sigma_r^3
};

cudaError_t launch_adjoint_lambda(const float* f, const float* gout, const float* Z, float* Lam, float* Dterm,
                                  double* partial, const GcParams& p, const AdjCoef& ac, size_t cs, cudaStream_t s);
cudaError_t launch_adjoint_assemble(const float* f, const float* Mch, const float* Dterm, float* gf, double* partial,
                                    const GcParams& p, const AdjCoef& ac, size_t cs, cudaStream_t s);
cudaError_t launch_adjoint_reduce(const double* partial, int n, double* out, cudaStream_t s);

}  // namespace bfgc
