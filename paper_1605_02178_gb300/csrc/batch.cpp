// Batches of independent images (declared in include/bfgc.h), in one of two modes:
//   * branches: the per-image forwards split over concurrent branches, run as one CUDA graph;
//   * persistent (tensor-core form): one launch of the batched row pass and one of the batched
//     column pass over a device work list of (image, tile) items (k_batch_tc.cu), captured in
//     a CUDA graph.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "bfgc_batch.h"
#include "bfgc_internal.h"

struct bf_gc_batch_s {
    std::vector<bf_gc_plan_t> plans;
    std::vector<int> branch_of;
    std::vector<std::vector<int>> members;      // images of each branch, in launch order
    std::vector<size_t> slice_off;              // workspace slice of each branch
    size_t ws_bytes = 0;
    // captured graph and the pointers it was captured with
    cudaGraphExec_t exec = nullptr;
    std::vector<const float*> cap_f;
    std::vector<float*> cap_out;
    void* cap_ws = nullptr;
    int captures = 0;
    std::vector<cudaStream_t> streams;          // [0] captures, [1..branches] the branches
    std::vector<cudaEvent_t> events;
    // persistent mode
    bool persistent = false;
    int a = 0, grid_rows = 0, grid_cols = 0;
    bool fp16 = false;
    bool any_pitch = false;                     // an image's rows are not a multiple of 16 bytes
    std::vector<bfgc::BatchImg> imgs;           // host copy of the image table
    std::vector<size_t> y_off;                  // channel buffer of each image in the workspace
    std::vector<int> row0, col0;
    size_t tab_bytes = 0;
    void* d_tab = nullptr;                      // device: images | row0 | col0
    void* h_tab = nullptr;                      // pinned staging copy of the same
};

namespace {

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

// Relative cost of one forward, for balancing the branches: the spatial bank dominates
// (eq. 7, about 2 (2R+1) C operations per pixel in the direct form; the tensor-core form's
// banded product is 2 (128 + 32 ceil(R/16)) C per pixel, on much faster units).
double plan_cost(const bf_gc_plan_s* p) {
    const double px = (double)p->H * p->W;
    if (p->form == BF_FORM_FUSED_TC) return px * p->C * (128.0 + 32.0 * std::ceil(p->R / 16.0)) * 0.05;
    if (p->form == BF_FORM_RECURSIVE) return px * p->C * 40.0;
    return px * p->C * (2.0 * p->R + 1.0);
}

void release_graph(bf_gc_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

// The Toeplitz words of an image (BatchImg::tt) in the channel storage's 16-bit format:
// tt[p][t] = (g(s - P), g(s + 1 - P)), s = 2t - 128 + p, g(d) = taps[|d|] for |d| <= R, else 0
void pack_toeplitz(bfgc::BatchImg& im, const float* taps, int R, int P, bool fp16) {
    auto g16 = [&](int d) -> uint32_t {
        const int ad = d < 0 ? -d : d;
        const float v = ad <= R ? taps[ad] : 0.0f;
        uint16_t bits;
        if (fp16) {
            const __half h = __float2half_rn(v);
            std::memcpy(&bits, &h, 2);
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            std::memcpy(&bits, &h, 2);
        }
        return bits;
    };
    for (int par = 0; par < 2; ++par)
        for (int t = 0; t < bfgc::kBatchTT; ++t) {
            const int s = 2 * t - 128 + par;
            im.tt[par][t] = g16(s - P) | (g16(s + 1 - P) << 16);
        }
}


// The persistent mode's forward: (re)write the image table when the pointers change, then the
// graph of [clear the counters, batched row pass, batched column pass].
bf_status persistent_forward(bf_gc_batch_s* b, const float* const* d_f, float* const* d_out, void* d_ws,
                             cudaStream_t stream) {
    const int count = (int)b->plans.size();
    const bool same = b->exec && b->cap_ws == d_ws && std::equal(b->cap_f.begin(), b->cap_f.end(), d_f) &&
                      std::equal(b->cap_out.begin(), b->cap_out.end(), d_out);
    if (same) return cudaGraphLaunch(b->exec, stream) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
    release_graph(b);
    for (int i = 0; i < count; ++i) {
        bfgc::BatchImg& im = b->imgs[i];
        const bf_gc_plan_s* p = b->plans[i];
        im.f = d_f[i];
        im.out = d_out[i];
        im.Y = (char*)d_ws + b->y_off[i];
        if (bfgc::encode_y_map(&im.ymap_st, im.Y, im.g, p->C, b->fp16, 64, p->C, im.g.r_rows, true) != cudaSuccess ||
            bfgc::encode_y_map(&im.ymap_ld, im.Y, im.g, p->C, b->fp16, 64, 1, im.g.kb_box_rows, true) != cudaSuccess)
            return BF_ERR_CUDA;
    }
    // table: images | row0 | col0, uploaded through the pinned copy in stream
    // order (the previous forward's kernels have read the old table before this copy runs)
    char* h = (char*)b->h_tab;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return BF_ERR_CUDA;   // the pinned copy is free
    size_t o = 0;
    auto put = [&](const void* src, size_t n) {
        std::memcpy(h + o, src, n);
        o += n;
    };
    put(b->imgs.data(), sizeof(bfgc::BatchImg) * count);
    const size_t o_row0 = o;
    put(b->row0.data(), sizeof(int) * b->row0.size());
    const size_t o_col0 = o;
    put(b->col0.data(), sizeof(int) * b->col0.size());
    if (cudaMemcpyAsync(b->d_tab, b->h_tab, b->tab_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return BF_ERR_CUDA;
    const char* t = (const char*)b->d_tab;
    bfgc::BatchWork wr{}, wc{};
    wr.imgs = wc.imgs = (const bfgc::BatchImg*)t;
    wr.nimg = wc.nimg = count;
    wr.wait_ns = wc.wait_ns = b->plans[0]->gp.wait_ns;
    wr.stall = wc.stall = b->plans[0]->gp.stall;
    wr.item0 = (const int*)(t + o_row0);
    wc.item0 = (const int*)(t + o_col0);
    wr.total = b->row0[count];
    wc.total = b->col0[count];
    DiagHeader* diag = (DiagHeader*)d_ws;
    if (b->streams.empty()) {
        b->streams.assign(1, nullptr);
        if (cudaStreamCreateWithFlags(&b->streams[0], cudaStreamNonBlocking) != cudaSuccess) return BF_ERR_CUDA;
    }
    cudaStream_t s0 = b->streams[0];
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BF_ERR_CUDA;
    bf_status st = BF_OK;
    if (cudaMemsetAsync(diag, 0, sizeof(DiagHeader), s0) != cudaSuccess ||
        bfgc::launch_rows_batch(wr, b->a, b->fp16, b->any_pitch, b->grid_rows, diag, s0) != cudaSuccess ||
        bfgc::launch_cols_batch(wc, b->a, b->fp16, b->any_pitch, b->grid_cols, diag, s0) != cudaSuccess)
        st = BF_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s0, &graph);
    if (st == BF_OK && ec != cudaSuccess) st = BF_ERR_CUDA;
    if (st == BF_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
        b->exec = nullptr;
        st = BF_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != BF_OK) return st;
    b->cap_f.assign(d_f, d_f + count);
    b->cap_out.assign(d_out, d_out + count);
    b->cap_ws = d_ws;
    ++b->captures;
    return cudaGraphLaunch(b->exec, stream) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

}  // namespace

extern "C" {

bf_status bf_gc_batch_create(int count, const bf_gc_plan_t* plans, int branches, bf_gc_batch_t* out) {
    if (out) *out = nullptr;
    if (!out || !plans || count < 1 || count > 65536 || branches < 1 || branches > 64) return BF_ERR_INVALID_ARG;
    std::vector<size_t> fwd(count, 0);
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || plans[i]->prof.enabled) return BF_ERR_INVALID_ARG;
        const bf_status st = bf_gc_workspace_size(plans[i], &fwd[i], nullptr);
        if (st != BF_OK) return st;
    }
    bf_gc_batch_s* b = new (std::nothrow) bf_gc_batch_s;
    if (!b) return BF_ERR_NOMEM;
    b->plans.assign(plans, plans + count);
    branches = std::min(branches, count);
    // longest processing time first: each image, costliest first, to the least loaded branch
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) cost[i] = plan_cost(plans[i]);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<double> load(branches, 0.0);
    b->branch_of.assign(count, 0);
    b->members.assign(branches, {});
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += cost[i];
        b->branch_of[i] = k;
        b->members[k].push_back(i);
    }
    // one workspace slice per branch, as large as its largest image needs
    b->slice_off.assign(branches, 0);
    size_t off = 0;
    for (int k = 0; k < branches; ++k) {
        size_t need = 256;
        for (int i : b->members[k]) need = std::max(need, round256(fwd[i]));
        b->slice_off[k] = off;
        off += need;
    }
    b->ws_bytes = off;
    *out = b;
    return BF_OK;
}

bf_status bf_gc_batch_create_persistent(int count, const bf_gc_plan_t* plans, bf_gc_batch_t* out) {
    if (out) *out = nullptr;
    if (!out || !plans || count < 1 || count > 65536) return BF_ERR_INVALID_ARG;
    int a = 1;
    for (int i = 0; i < count; ++i) {
        const bf_gc_plan_s* p = plans[i];
        if (!p || p->prof.enabled) return BF_ERR_INVALID_ARG;
        if (p->form != BF_FORM_FUSED_TC || p->tile_w != 0 || p->precision != plans[0]->precision ||
            (p->precision != BF_PREC_BF16 && p->precision != BF_PREC_FP16) || p->R > 16 * bfgc::kBatchMaxA ||
            !bfgc::tc_supported(p->R, p->C))
            return BF_ERR_UNSUPPORTED;
        a = std::max(a, (p->R + 15) / 16);
    }
    bf_gc_batch_s* b = new (std::nothrow) bf_gc_batch_s;
    if (!b) return BF_ERR_NOMEM;
    b->persistent = true;
    b->plans.assign(plans, plans + count);
    b->branch_of.assign(count, 0);
    b->a = a;
    b->fp16 = plans[0]->precision == BF_PREC_FP16;
    for (int i = 0; i < count; ++i) b->any_pitch = b->any_pitch || (plans[i]->W & 3) != 0;
    b->imgs.resize(count);
    b->y_off.resize(count);
    std::vector<int> nrow(count), ncol(count);
    size_t off = 256;                                      // DiagHeader of the batch
    long long rows_total = 0, cols_total = 0;
    for (int i = 0; i < count; ++i) {
        const bf_gc_plan_s* p = plans[i];
        bfgc::BatchImg& im = b->imgs[i];
        std::memset(&im, 0, sizeof(im));
        im.g = bfgc::tc_geometry(p->H, p->W, 16 * a, p->C);
        im.p = p->gp;
        im.p.refine = nullptr;                             // the FP32 guard of eq. (10)
        im.R = p->R;
        pack_toeplitz(im, p->taps.g, p->R, im.g.P, b->fp16);
        b->y_off[i] = off;
        off += round256((size_t)p->C * im.g.Hp * im.g.Wp * 2);
        nrow[i] = ((im.g.Wp + 127) / 128) * ((im.g.Hp + im.g.r_rows - 1) / im.g.r_rows);
        ncol[i] = (im.g.Wp / 64) * ((im.g.Hp - 2 * im.g.P) / 128);
        rows_total += nrow[i];
        cols_total += ncol[i];
    }
    if (rows_total >= (1ll << 30) || cols_total >= (1ll << 30)) {
        delete b;
        return BF_ERR_UNSUPPORTED;
    }
    b->ws_bytes = off;
    b->row0.assign(count + 1, 0);
    b->col0.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        b->row0[i + 1] = b->row0[i] + nrow[i];
        b->col0[i + 1] = b->col0[i] + ncol[i];
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    b->grid_rows = (int)std::min<long long>(sms, (rows_total + bfgc::kBatchRowChunk - 1) / bfgc::kBatchRowChunk);
    b->grid_cols = (int)std::min<long long>(sms, (cols_total + bfgc::kBatchColChunk - 1) / bfgc::kBatchColChunk);
    b->tab_bytes = sizeof(bfgc::BatchImg) * count + sizeof(int) * (b->row0.size() + b->col0.size());
    if (cudaMalloc(&b->d_tab, b->tab_bytes) != cudaSuccess || cudaMallocHost(&b->h_tab, b->tab_bytes) != cudaSuccess) {
        bf_gc_batch_destroy(b);
        return BF_ERR_CUDA;
    }
    *out = b;
    return BF_OK;
}

bf_status bf_gc_batch_workspace_size(bf_gc_batch_t b, size_t* bytes) {
    if (!b || !bytes) return BF_ERR_INVALID_ARG;
    *bytes = b->ws_bytes;
    return BF_OK;
}

bf_status bf_gc_batch_info(bf_gc_batch_t b, int* branch_of, int* captures) {
    if (!b) return BF_ERR_INVALID_ARG;
    if (branch_of) std::copy(b->branch_of.begin(), b->branch_of.end(), branch_of);
    if (captures) *captures = b->captures;
    return BF_OK;
}

bf_status bf_gc_batch_forward(bf_gc_batch_t b, const float* const* d_f, float* const* d_out, void* d_ws,
                              size_t ws_bytes, bf_stream_t stream) {
    if (!b || !d_f || !d_out) return BF_ERR_INVALID_ARG;
    if (!d_ws || ((uintptr_t)d_ws & 255) || ws_bytes < b->ws_bytes) return BF_ERR_WORKSPACE;
    const int count = (int)b->plans.size(), nbr = (int)b->members.size();
    for (int i = 0; i < count; ++i)
        if (!d_f[i] || !d_out[i] || ((uintptr_t)d_f[i] & 15) || ((uintptr_t)d_out[i] & 15)) return BF_ERR_INVALID_ARG;
    if (b->persistent) return persistent_forward(b, d_f, d_out, d_ws, (cudaStream_t)stream);
    const bool same = b->exec && b->cap_ws == d_ws && std::equal(b->cap_f.begin(), b->cap_f.end(), d_f) &&
                      std::equal(b->cap_out.begin(), b->cap_out.end(), d_out);
    if (!same) {
        release_graph(b);
        if (b->streams.empty()) {
            b->streams.assign(nbr + 1, nullptr);
            b->events.assign(nbr + 1, nullptr);
            for (int k = 0; k <= nbr; ++k) {
                if (cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&b->events[k], cudaEventDisableTiming) != cudaSuccess)
                    return BF_ERR_CUDA;
            }
        }
        cudaStream_t s0 = b->streams[0];
        if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BF_ERR_CUDA;
        bf_status st = BF_OK;
        // fork: every branch waits for the capture origin
        if (cudaEventRecord(b->events[0], s0) != cudaSuccess) st = BF_ERR_CUDA;
        for (int k = 0; k < nbr && st == BF_OK; ++k) {
            cudaStream_t sk = b->streams[k + 1];
            if (cudaStreamWaitEvent(sk, b->events[0], 0) != cudaSuccess) {
                st = BF_ERR_CUDA;
                break;
            }
            char* ws = (char*)d_ws + b->slice_off[k];
            const size_t slice = (k + 1 < nbr ? b->slice_off[k + 1] : b->ws_bytes) - b->slice_off[k];
            for (int i : b->members[k]) {
                st = bf_gc_forward(b->plans[i], d_f[i], d_out[i], ws, slice, (bf_stream_t)sk);
                if (st != BF_OK) break;
            }
            // join: the origin waits for every branch
            if (st == BF_OK && (cudaEventRecord(b->events[k + 1], sk) != cudaSuccess ||
                                cudaStreamWaitEvent(s0, b->events[k + 1], 0) != cudaSuccess))
                st = BF_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s0, &graph);
        if (st == BF_OK && ec != cudaSuccess) st = BF_ERR_CUDA;
        if (st == BF_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) {
            b->exec = nullptr;
            st = BF_ERR_CUDA;
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != BF_OK) return st;
        b->cap_f.assign(d_f, d_f + count);
        b->cap_out.assign(d_out, d_out + count);
        b->cap_ws = d_ws;
        ++b->captures;
    }
    return cudaGraphLaunch(b->exec, (cudaStream_t)stream) == cudaSuccess ? BF_OK : BF_ERR_CUDA;
}

void bf_gc_batch_destroy(bf_gc_batch_t b) {
    if (!b) return;
    release_graph(b);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->events)
        if (e) cudaEventDestroy(e);
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->h_tab) cudaFreeHost(b->h_tab);
    delete b;
}

}  // extern "C"
