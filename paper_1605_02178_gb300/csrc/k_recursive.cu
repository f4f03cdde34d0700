// Recursive stand-in for the spatial Gaussian of eq. (7) (the paper computes eq. (7) "using
// separability and recursion" without fixing the recursion): the third-order causal +
// anti-causal filter of Young and van Vliet (Signal Processing 44, 1995), applied along the
// rows, then along the columns, of every channel plane.
//
// Each line of n samples is extended by P samples of half-sample mirror on each side; the
// causal pass
//     w[q] = B x[q] + a1 w[q-1] + a2 w[q-2] + a3 w[q-3]
// starts from the steady state of the first extended sample, the anti-causal pass
//     y[q] = B w[q] + a1 y[q+1] + a2 y[q+2] + a3 y[q+3]
// from the steady state of the last causal output; the central n outputs are kept.  The
// causal outputs of the trailing P extended samples go to a per-line scratch area.
//
// Arithmetic.  For large sigma the recursion has a DC gain of 1/B in the hundreds, so FP32
// rounding injected into the state is amplified by that much.  The state is therefore
// advanced in increment form, using a1 = 1 - B - a2 - a3 (unit DC gain):
//     w[q] = w[q-1] + B (x - w[q-1]) + a2 (w[q-2] - w[q-1]) + a3 (w[q-3] - w[q-1]),
// with each state value kept as an unevaluated sum hi + lo of two floats (the increment is
// added with an error-free two-sum), so the only rounding left per step is on the small
// increment.
#include "bfgc_common.cuh"
#include "bfgc_recursive.h"

namespace bfgc {

struct IirState {
    float h1, l1, h2, l2, h3, l3;   // w[q-1], w[q-2], w[q-3] as hi + lo
    __device__ __forceinline__ void init(float v) {
        h1 = h2 = h3 = v;
        l1 = l2 = l3 = 0.0f;
    }
    // advance with input x; returns the new value rounded to float
    __device__ __forceinline__ float step(const IirCoef& c, float x) {
        const float d = c.B * ((x - h1) - l1) + c.a2 * ((h2 - h1) + (l2 - l1)) + c.a3 * ((h3 - h1) + (l3 - l1));
        const float s = h1 + d;                       // two-sum of h1 and d
        const float bb = s - h1;
        const float err = (h1 - (s - bb)) + (d - bb);
        const float lo = err + l1;
        const float hi = s + lo;                      // renormalise
        const float nlo = lo - (hi - s);
        h3 = h2; l3 = l2;
        h2 = h1; l2 = l1;
        h1 = hi; l1 = nlo;
        return hi;
    }
};

// ---------------------------------------------------------------------------------------
// Rows: one warp filters 32 rows of one plane, 32 columns at a time through a transposed
// shared-memory tile (coalesced loads and stores, conflict-free column walks).
constexpr int IR_TILE = 32;

__global__ void __launch_bounds__(32, 16) k_iir_rows(const float* __restrict__ X, float* __restrict__ Y,
                                                 float* __restrict__ tail, const GcParams p, const IirCoef c,
                                                 size_t cs) {
    __shared__ float tile[IR_TILE][IR_TILE + 1];
    const int lane = threadIdx.x;
    const int n = p.W, P = c.P;
    const int row0 = blockIdx.x * IR_TILE, plane = blockIdx.y;
    const int myrow = row0 + lane;
    const bool live = myrow < p.H;
    const float* src = X + (size_t)plane * cs;
    float* dst = Y + (size_t)plane * cs;
    const int ext = n + 2 * P;
    const int chunks = (ext + IR_TILE - 1) / IR_TILE;

    IirState st;
    {
        const float x0 = live ? src[(size_t)myrow * n + mirror(-P, n)] : 0.0f;
        st.init(x0);
    }
    // causal: chunk k covers extended positions q = 32k .. 32k+31 (x index q - P)
    for (int k = 0; k < chunks; ++k) {
        float v[IR_TILE];                             // all 32 loads in flight before any store
#pragma unroll
        for (int r = 0; r < IR_TILE; ++r) {          // load: row r, lane = column
            const int row = row0 + r;
            const int q = k * IR_TILE + lane, xi = q - P;
            v[r] = 0.0f;
            if (row < p.H && q < ext) v[r] = src[(size_t)row * n + ((unsigned)xi < (unsigned)n ? xi : mirror(xi, n))];
        }
#pragma unroll
        for (int r = 0; r < IR_TILE; ++r) tile[r][lane] = v[r];
        __syncwarp();
        for (int j = 0; j < IR_TILE; ++j) {           // walk my row
            const int q = k * IR_TILE + j;
            if (q < ext) tile[lane][j] = st.step(c, tile[lane][j]);
        }
        __syncwarp();
        for (int r = 0; r < IR_TILE; ++r) {          // store causal output (image part / tail)
            const int row = row0 + r;
            const int q = k * IR_TILE + lane, xi = q - P;
            if (row < p.H && q < ext) {
                if (xi >= 0 && xi < n) dst[(size_t)row * n + xi] = tile[r][lane];
                else if (xi >= n) tail[((size_t)plane * p.H + row) * (size_t)P + (xi - n)] = tile[r][lane];
            }
        }
        __syncwarp();
    }
    // anti-causal: from q = ext-1 down to P, chunks walked backwards
    {
        const float wl = st.h1;
        st.init(wl);
    }
    for (int k = chunks - 1; k >= 0; --k) {
        float v[IR_TILE];
#pragma unroll
        for (int r = 0; r < IR_TILE; ++r) {
            const int row = row0 + r;
            const int q = k * IR_TILE + lane, xi = q - P;
            v[r] = 0.0f;
            if (row < p.H && q < ext && xi >= 0)
                v[r] = xi < n ? dst[(size_t)row * n + xi] : tail[((size_t)plane * p.H + row) * (size_t)P + (xi - n)];
        }
#pragma unroll
        for (int r = 0; r < IR_TILE; ++r) tile[r][lane] = v[r];
        __syncwarp();
        for (int j = IR_TILE - 1; j >= 0; --j) {
            const int q = k * IR_TILE + j;
            if (q < ext && q >= P) tile[lane][j] = st.step(c, tile[lane][j]);
        }
        __syncwarp();
        for (int r = 0; r < IR_TILE; ++r) {
            const int row = row0 + r;
            const int q = k * IR_TILE + lane, xi = q - P;
            if (row < p.H && q < ext && xi >= 0 && xi < n) dst[(size_t)row * n + xi] = tile[r][lane];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------
// Columns: one thread per column (consecutive threads, consecutive columns: coalesced).
__global__ void __launch_bounds__(128) k_iir_cols(const float* __restrict__ X, float* __restrict__ Y,
                                                  float* __restrict__ tail, const GcParams p, const IirCoef c,
                                                  size_t cs) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.W) return;
    const int plane = blockIdx.y, n = p.H, P = c.P, W = p.W;
    const float* x = X + (size_t)plane * cs + col;
    float* y = Y + (size_t)plane * cs + col;
    float* tl = tail + ((size_t)plane * W + col) * (size_t)P;
    const int ext = n + 2 * P;
    constexpr int B = 16;                             // loads issued together per block of steps
    IirState st;
    st.init(x[(size_t)mirror(-P, n) * W]);
    for (int q0 = 0; q0 < ext; q0 += B) {
        float v[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = q0 + j - P;
            v[j] = q0 + j < ext ? x[(size_t)((unsigned)k < (unsigned)n ? k : mirror(k, n)) * W] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = q0 + j - P;
            if (q0 + j < ext) {
                const float w = st.step(c, v[j]);
                if (k >= 0 && k < n) y[(size_t)k * W] = w;
                else if (k >= n) tl[k - n] = w;
            }
        }
    }
    st.init(st.h1);
    for (int q0 = ext - 1; q0 >= P; q0 -= B) {        // q = q0, q0-1, ..., down to P
        float v[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = q0 - j - P;
            v[j] = q0 - j >= P ? (k >= n ? tl[k - n] : y[(size_t)k * W]) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = q0 - j - P;
            if (q0 - j >= P) {
                const float r = st.step(c, v[j]);
                if (k < n) y[(size_t)k * W] = r;
            }
        }
    }
}

cudaError_t launch_iir(int axis, const float* X, float* Y, float* tail, const GcParams& p, const IirCoef& c,
                       size_t cs, int planes, cudaStream_t s) {
    if (axis == 0) {
        dim3 grid((p.H + IR_TILE - 1) / IR_TILE, planes);
        k_iir_rows<<<grid, IR_TILE, 0, s>>>(X, Y, tail, p, c, cs);
    } else {
        dim3 grid((p.W + 127) / 128, planes);
        k_iir_cols<<<grid, 128, 0, s>>>(X, Y, tail, p, c, cs);
    }
    return cudaGetLastError();
}

}  // namespace bfgc
