// Batches of independent images: the per-image forwards split over concurrent branches and
// run as one CUDA graph (declared in include/bfgc.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <numeric>
#include <vector>

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
        if (!d_f[i] || !d_out[i]) return BF_ERR_INVALID_ARG;
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
    delete b;
}

}  // extern "C"
