// Geometry and launchers of the fused tensor-core form (k_rows_tc.cu: row pass with the
// Toeplitz operand in tensor memory, the default; k_umma.cu: row pass with the Toeplitz
// operand in shared memory and a chosen tile width; k_cols_tc.cu: column pass + ratio with two
// channels per MMA step, for ceil(R/16) <= 7; k_tc.cu: column pass + ratio with one channel
// per step, for ceil(R/16) = 8, and the geometry).
#pragma once

#include <cuda.h>

#include "bfgc_internal.h"

namespace bfgc {

// Row-filtered channel buffer Y[p][c][x]: Hp padded rows, each holding the C channel rows of
// Wp columns, 2-byte elements.  Padded row p holds image row p - P (mirrored into [0, H));
// P = 16a rows of margin above and below, Hp = round_up(H, 128) + 2P, Wp = round_up(W, 64).
struct TcGeom {
    int a;            // ceil(R / 16): Toeplitz k-blocks on each side of an output block
    int P, Hp, Wp;
    int kb_stages;    // TMA ring depth of the column pass kernel
    int kb_box_rows;  // rows per TMA box (tile rows or half of them)
    // tcgen05 row pass with the Toeplitz operand in shared memory (k_umma.cu)
    int u_rows;       // padded rows per tile: floor(128 / C) (fewer if the octets do not fit)
    int u_tw;         // output columns per tile: 64, 128 or 256 (default 256, or 64 when a > 4)
    int u_hb;         // 64-column halo blocks on each side: ceil(a / 4)
    int u_nkb;        // 64-column K-blocks of the channel operand: u_tw / 64 + 2 u_hb
    int u_kbb;        // 64-column K-blocks of the Toeplitz operand: ceil((64 + 32a) / 64)
    // tcgen05 row pass with the Toeplitz operand in tensor memory (k_rows_tc.cu)
    int r_rows;       // padded rows per tile: floor(128 / C) (fewer if the octets do not fit)
    int r_stages;     // channel-buffer ring depth (2 .. 4)
    int r_stg;        // staging tiles of the drain's TMA stores (1 .. 3)
    int r_np;         // product rows per tile (the MMA's N): r_rows C rounded up to 16
    // column pass with channel pairs (k_cols_tc.cu); 0 when a > 7 (one channel per step, k_tc.cu)
    int vp_stages;    // ring depth, stages of two channel tiles (2 .. 4)
};

// tw: row-pass tile width (64, 128 or 256; 128 and 256 only for a <= 4), 0 for the default
TcGeom tc_geometry(int H, int W, int R, int C, int tw = 0);
size_t tc_workspace_bytes(const TcGeom& g, int C);
bool tc_supported(int R, int C);
size_t umma_smem_bytes(const TcGeom& g);
int umma_max_octets();
int rows_tc_max_octets();
size_t rows_tc_stage_bytes(int a, int np);
size_t rows_tc_stg_bytes(int np);
size_t rows_tc_smem_bytes(const TcGeom& g);
// The driver's cuTensorMapEncodeTiled, looked up once (null if unavailable)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn();
// Tensor map of the row-filtered buffer Y[p][c][x] (3-D: x, c, p) with the given box
cudaError_t encode_y_map(CUtensorMap* map, void* Y, const TcGeom& g, int C, bool fp16, int box_x, int box_c,
                         int box_rows, bool swizzle128);
cudaError_t launch_build_hpass_tc(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                  bool fp16, DiagHeader* diag, cudaStream_t s);
cudaError_t launch_build_hpass_umma(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                    bool fp16, DiagHeader* diag, cudaStream_t s);
int vp_stages_for(int a);
size_t vp_smem_bytes(const TcGeom& g);
cudaError_t launch_vpass_combine_pairs(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                       const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s);
cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s);

}  // namespace bfgc
