// Persistent batched tensor-core forward (k_batch_tc.cu, batch.cpp): one launch of the row pass
// and one of the column pass over a device work list of (image, tile) items of many images.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "bfgc_internal.h"
#include "bfgc_tc.h"

namespace bfgc {

// Largest window block count a = ceil(R / 16) of the persistent batch: two Toeplitz operands
// (one per image in flight, 64 + 16a <= 128 tensor-memory columns each) beside two 128-column
// accumulator buffers fill the 512 columns.
constexpr int kBatchMaxA = 4;
// Packed Toeplitz words of an image (see BatchImg::tt): 2 lane parities x 192 words
constexpr int kBatchTT = 192;

// One image of the batch.  Every image is laid out at the batch's a (its padded rows and the
// tile geometry use P = 16a), with its own taps g(0..R), zero beyond its R: the banded
// products then equal those of the image's own a.  (Aligned as its tensor maps.)
struct BatchImg {
    CUtensorMap ymap_st;          // row pass: Y stores, box {64 columns, C channels, r_rows rows}
    CUtensorMap ymap_ld;          // column pass: Y loads, box {64 columns, 1 channel, kb_box_rows}
    GcParams p;                   // H, W, N, C, R, u-mapping, coefficients, guard (refine = null)
    TcGeom g;                     // geometry at the batch's a
    const float* f;
    float* out;
    void* Y;
    int R;
    // The Toeplitz operand as 16-bit pairs: lane i, tensor-memory column c holds
    // (g(2c - P - i), g(2c + 1 - P - i)) = tt[i & 1][c + (128 - i - (i & 1)) / 2], i.e.
    // tt[p][t] = (g(s - P), g(s + 1 - P)) with s = 2t - 128 + p (g zero beyond R).
    uint32_t tt[2][kBatchTT];
};

// A launch's view of the work list: items of image i are item0[i] .. item0[i + 1] - 1 (row-pass
// tiles or column-pass tiles in the per-image kernels' order), `total` in all.  The list is cut
// into chunks of consecutive items (kBatchRowChunk, kBatchColChunk); CTA b takes chunks b, b + grid, b + 2 grid, ...,
// so that the CTAs work on neighbouring tiles at the same time (shared halo rows meet in L2,
// and the writes stay in a narrow address range).
struct BatchWork {
    const BatchImg* imgs;
    const int* item0;
    int nimg, total;
    unsigned long long wait_ns;
    // test of the bounded waits (BF_OPT_STALL of the first plan): 1 = the row pass's first
    // build group never hands over its first tile, 2 = the column pass never loads its first
    // stage; nothing asynchronous is outstanding for the withheld step
    int stall;
};
// Chunk sizes of the two passes' work lists (consecutive row-pass / column-pass tiles)
constexpr int kBatchRowChunk = 4, kBatchColChunk = 2;

// Shared-memory ring of the batched row pass at window block count a: stages of KB K-blocks of
// 128 product rows, staging tiles of 128 rows (the largest product-row count of any image).
void rows_batch_ring(int a, int* stages, int* staging);
size_t rows_batch_smem(int a);
size_t cols_batch_smem(int a);
int cols_batch_stages(int a);

// any_pitch: some image's rows are not a multiple of 16 bytes (W % 4 != 0); such a batch takes
// the instantiations that also use 8- and 16-byte accesses inside those rows
cudaError_t launch_rows_batch(const BatchWork& w, int a, bool fp16, bool any_pitch, int grid, DiagHeader* diag,
                              cudaStream_t s);
cudaError_t launch_cols_batch(const BatchWork& w, int a, bool fp16, bool any_pitch, int grid, DiagHeader* diag,
                              cudaStream_t s);

}  // namespace bfgc
