// Geometry and launchers of the fused tensor-core form (k_tc.cu).
#pragma once

#include "bfgc_internal.h"

namespace bfgc {

// Row-filtered channel buffer Y[c][p][x]: C planes of Hp padded rows by Wp columns, 2-byte
// elements.  Padded row p holds image row p - P (mirrored into [0, H)); P = 16a rows of
// margin above and below, Hp = round_up(H, 64) + 2P, Wp = round_up(W, 64).
struct TcGeom {
    int a;            // ceil(R / 16): Toeplitz k-blocks on each side of an output block
    int P, Hp, Wp;
    int ka_rows;      // padded rows per tile of the build + row pass kernel
    int kb_stages;    // TMA ring depth of the column pass kernel
    int kb_box_rows;  // rows per TMA box (tile rows or half of them)
};

TcGeom tc_geometry(int H, int W, int R, int C);
size_t tc_workspace_bytes(const TcGeom& g, int C);
bool tc_supported(int R, int C);
cudaError_t launch_build_hpass_tc(const float* f, void* Y, const GcParams& p, const Taps& t, const TcGeom& g,
                                  bool fp16, cudaStream_t s);
cudaError_t launch_vpass_combine_tc(const float* f, void* Y, float* out, const GcParams& p, const Taps& t,
                                    const TcGeom& g, bool fp16, DiagHeader* diag, cudaStream_t s);

}  // namespace bfgc
