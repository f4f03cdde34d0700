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
#include <algorithm>
#include <cmath>

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
// Rows: one warp filters 32 rows of one plane over one segment of the extended line, 32
// columns at a time through a transposed shared-memory tile (coalesced loads, copied straight
// into shared memory with cp.async, coalesced stores, conflict-free column walks); four such
// warps to a block.  A line is split into segments that run in parallel (a line's
// recursion is sequential, and C x H lines leave too few warps to hide its latency): the
// causal pass of a segment other than the first starts `warm` samples before the segment from
// the steady state of the sample there, and the anti-causal pass of a segment other than the
// last `warm` samples after it from the steady state of the causal output there.  The state
// error this leaves decays like the recursion's impulse response; `warm` is where that response
// has fallen below 1e-8 of its peak (from the coefficients, on the host), so the segments agree
// with the unsegmented recursion to that level.  The causal pass reads X and writes Y (the tail
// of trailing pad samples to `tail`); the anti-causal pass reads Y and writes X, so that no
// segment overwrites samples another segment still reads.
constexpr int IR_TILE = 32;
constexpr int IR_WARPS = 4;                           // warps per block, each with its own 32 rows

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" :: "r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

__global__ void __launch_bounds__(IR_TILE * IR_WARPS, 8) k_iir_rows_causal(const float* __restrict__ X,
                                                                       float* __restrict__ Y,
                                                                       float* __restrict__ tail, const GcParams p,
                                                                       const IirCoef c, size_t cs, int seg_len,
                                                                       int warm) {
    __shared__ float tiles[IR_WARPS][IR_TILE][IR_TILE + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float(*tile)[IR_TILE + 1] = tiles[wid];
    const int n = p.W, P = c.P, ext = n + 2 * P;
    const int row0 = (blockIdx.x * IR_WARPS + wid) * IR_TILE, plane = blockIdx.y;
    const int qs = blockIdx.z * seg_len;
    if (qs >= ext || row0 >= p.H) return;
    const int qe = min(ext, qs + seg_len);
    const int q0 = blockIdx.z == 0 ? 0 : max(0, qs - warm);
    const int myrow = row0 + lane;
    const float* src = X + (size_t)plane * cs;
    float* dst = Y + (size_t)plane * cs;
    auto xptr = [&](int row, int q) {
        const int xi = q - P;
        return src + (size_t)row * n + ((unsigned)xi < (unsigned)n ? xi : mirror(xi, n));
    };

    IirState st;
    st.init(myrow < p.H ? *xptr(myrow, q0) : 0.0f);
    for (int qc = q0; qc < qe; qc += IR_TILE) {     // chunk: positions qc .. qc + 31
        // load: row r, lane = position, straight into shared memory
        for (int r = 0; r < IR_TILE; ++r) {
            const int row = row0 + r, q = qc + lane;
            if (row < p.H && q < qe) cp_async4(&tile[r][lane], xptr(row, q));
            else tile[r][lane] = 0.0f;
        }
        cp_async_wait_all();
        __syncwarp();
        for (int j = 0; j < IR_TILE; ++j)            // walk my row
            if (qc + j < qe) tile[lane][j] = st.step(c, tile[lane][j]);
        __syncwarp();
        for (int r = 0; r < IR_TILE; ++r) {          // store the segment's causal outputs
            const int row = row0 + r, q = qc + lane, xi = q - P;
            if (row < p.H && q >= qs && q < qe) {
                if (xi >= 0 && xi < n) dst[(size_t)row * n + xi] = tile[r][lane];
                else if (xi >= n) tail[((size_t)plane * p.H + row) * (size_t)P + (xi - n)] = tile[r][lane];
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(IR_TILE * IR_WARPS, 8) k_iir_rows_anti(const float* __restrict__ Y,
                                                                     float* __restrict__ X,
                                                                     const float* __restrict__ tail,
                                                                     const GcParams p, const IirCoef c, size_t cs,
                                                                     int seg_len, int warm) {
    __shared__ float tiles[IR_WARPS][IR_TILE][IR_TILE + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float(*tile)[IR_TILE + 1] = tiles[wid];
    const int n = p.W, P = c.P, ext = n + 2 * P;
    const int row0 = (blockIdx.x * IR_WARPS + wid) * IR_TILE, plane = blockIdx.y;
    const int qs = blockIdx.z * seg_len;
    if (qs >= ext || row0 >= p.H) return;
    const int qe = min(ext, qs + seg_len);
    if (qe <= P) return;                              // the segment lies in the left pad
    const int lo = max(qs, P);                        // outputs for lo .. qe - 1 (image part)
    const int q1 = qe == ext ? ext - 1 : min(ext - 1, qe - 1 + warm);
    const int myrow = row0 + lane;
    const float* w = Y + (size_t)plane * cs;
    float* dst = X + (size_t)plane * cs;
    auto wptr = [&](int row, int q) {                 // causal output at extended position q >= P
        const int xi = q - P;
        return xi < n ? w + (size_t)row * n + xi : tail + ((size_t)plane * p.H + row) * (size_t)P + (xi - n);
    };

    IirState st;
    st.init(myrow < p.H ? *wptr(myrow, q1) : 0.0f);
    for (int qc = q1 - (IR_TILE - 1); qc + IR_TILE - 1 >= lo; qc -= IR_TILE) {   // positions qc .. qc + 31
        for (int r = 0; r < IR_TILE; ++r) {
            const int row = row0 + r, q = qc + lane;
            if (row < p.H && q >= lo && q <= q1) cp_async4(&tile[r][lane], wptr(row, q));
            else tile[r][lane] = 0.0f;
        }
        cp_async_wait_all();
        __syncwarp();
        for (int j = IR_TILE - 1; j >= 0; --j) {
            const int q = qc + j;
            if (q >= lo && q <= q1) tile[lane][j] = st.step(c, tile[lane][j]);
        }
        __syncwarp();
        for (int r = 0; r < IR_TILE; ++r) {
            const int row = row0 + r, q = qc + lane, xi = q - P;
            if (row < p.H && q >= lo && q < qe && xi < n) dst[(size_t)row * n + xi] = tile[r][lane];
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

// Samples after which the recursion's impulse response stays below 1e-8 of its peak (the
// warm-up of a segment), from the coefficients, in double
int iir_warmup(const IirCoef& c) {
    const double a1 = c.a1, a2 = c.a2, a3 = c.a3;
    double h1 = 1.0, h2 = 0.0, h3 = 0.0, peak = 1.0;
    int last = 0;
    for (int t = 1; t < 1 << 16; ++t) {
        const double h = a1 * h1 + a2 * h2 + a3 * h3;
        h3 = h2;
        h2 = h1;
        h1 = h;
        peak = std::max(peak, std::fabs(h));
        if (std::fabs(h) > 1e-8 * peak) last = t;
        else if (t > 4 * last + 64) break;           // decayed for good
    }
    return last + 1;
}

cudaError_t launch_iir(int axis, float* X, float* Y, float* tail, const GcParams& p, const IirCoef& c, size_t cs,
                       int planes, cudaStream_t s) {
    if (axis == 0) {
        // segments of at least three warm-ups (the overhead stays near a third) and at most 16
        const int ext = p.W + 2 * c.P, warm = iir_warmup(c);
        int seg_len = std::max({3 * warm, 256, (ext + 15) / 16});
        seg_len = (seg_len + IR_TILE - 1) / IR_TILE * IR_TILE;
        const int nseg = (ext + seg_len - 1) / seg_len;
        dim3 grid(((p.H + IR_TILE - 1) / IR_TILE + IR_WARPS - 1) / IR_WARPS, planes, nseg);
        k_iir_rows_causal<<<grid, IR_TILE * IR_WARPS, 0, s>>>(X, Y, tail, p, c, cs, seg_len, warm);
        k_iir_rows_anti<<<grid, IR_TILE * IR_WARPS, 0, s>>>(Y, X, tail, p, c, cs, seg_len, warm);
    } else {
        dim3 grid((p.W + 127) / 128, planes);
        k_iir_cols<<<grid, 128, 0, s>>>(X, Y, tail, p, c, cs);
    }
    return cudaGetLastError();
}

}  // namespace bfgc
