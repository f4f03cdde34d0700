// Recursive (Young-van Vliet) spatial passes, k_recursive.cu.
#pragma once

#include "bfgc_internal.h"

namespace bfgc {

struct IirCoef {
    int P;                   // mirror samples added on each side of a line (= R)
    float B, a1, a2, a3;     // w[q] = B x[q] + a1 w[q-1] + a2 w[q-2] + a3 w[q-3]
};

// axis 0: along rows (lines = rows): X in, result in X (Y is overwritten on the way);
// axis 1: along columns: X in, result in Y.  tail: planes * lines * P floats.
cudaError_t launch_iir(int axis, float* X, float* Y, float* tail, const GcParams& p, const IirCoef& c, size_t cs,
                       int planes, cudaStream_t s);

}  // namespace bfgc
