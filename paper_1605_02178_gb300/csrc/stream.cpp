// Streaming forward of many images held in host memory (declared in include/bfgc.h): the
// uploads, the filtering and the downloads of consecutive images overlap on three internal
// streams ordered by events, over two device slots.
#include <cuda_runtime.h>

#include <cstdint>

#include "bfgc_internal.h"

namespace {

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

struct StreamRes {
    cudaStream_t up = nullptr, run = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, in_ready[2] = {}, run_done[2] = {}, out_done[2] = {};
    ~StreamRes() {
        for (cudaStream_t s : {up, run, down})
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : {start, in_ready[0], in_ready[1], run_done[0], run_done[1], out_done[0], out_done[1]})
            if (e) cudaEventDestroy(e);
    }
    bool make() {
        for (cudaStream_t* s : {&up, &run, &down})
            if (cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess) return false;
        for (cudaEvent_t* e : {&start, &in_ready[0], &in_ready[1], &run_done[0], &run_done[1], &out_done[0], &out_done[1]})
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
        return true;
    }
};

}  // namespace

extern "C" {

bf_status bf_gc_stream_bytes(bf_gc_plan_t p, size_t* bytes) {
    if (!p || !bytes) return BF_ERR_INVALID_ARG;
    size_t fwd = 0;
    const bf_status st = bf_gc_workspace_size(p, &fwd, nullptr);
    if (st != BF_OK) return st;
    const size_t img = round256((size_t)p->H * p->W * sizeof(float));
    *bytes = 4 * img + round256(fwd);
    return BF_OK;
}

bf_status bf_gc_forward_host_stream(bf_gc_plan_t p, int count, const float* const* h_f, float* const* h_out,
                                    void* d_scratch, size_t scratch_bytes, bf_stream_t stream) {
    if (!p || count < 1 || !h_f || !h_out) return BF_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!h_f[i] || !h_out[i]) return BF_ERR_INVALID_ARG;
    size_t need = 0;
    bf_status st = bf_gc_stream_bytes(p, &need);
    if (st != BF_OK) return st;
    if (!d_scratch || ((uintptr_t)d_scratch & 255) || scratch_bytes < need) return BF_ERR_WORKSPACE;
    const size_t bytes = (size_t)p->H * p->W * sizeof(float), img = round256(bytes);
    char* base = static_cast<char*>(d_scratch);
    float* d_in[2] = {reinterpret_cast<float*>(base), reinterpret_cast<float*>(base + img)};
    float* d_out[2] = {reinterpret_cast<float*>(base + 2 * img), reinterpret_cast<float*>(base + 3 * img)};
    void* ws = base + 4 * img;
    const size_t ws_bytes = scratch_bytes - 4 * img;

    StreamRes r;
    if (!r.make()) return BF_ERR_CUDA;
    // everything already queued on the caller's stream (e.g. the scratch's last use) first
    bool ok = cudaEventRecord(r.start, (cudaStream_t)stream) == cudaSuccess &&
              cudaStreamWaitEvent(r.up, r.start, 0) == cudaSuccess &&
              cudaStreamWaitEvent(r.run, r.start, 0) == cudaSuccess;
    for (int i = 0; i < count && ok; ++i) {
        const int k = i & 1;
        // upload image i into slot k once the filtering of image i - 2 has read it
        if (i >= 2) ok = ok && cudaStreamWaitEvent(r.up, r.run_done[k], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(d_in[k], h_f[i], bytes, cudaMemcpyHostToDevice, r.up) == cudaSuccess &&
             cudaEventRecord(r.in_ready[k], r.up) == cudaSuccess;
        // filter it into output slot k once the download of image i - 2 has read that slot
        ok = ok && cudaStreamWaitEvent(r.run, r.in_ready[k], 0) == cudaSuccess;
        if (i >= 2) ok = ok && cudaStreamWaitEvent(r.run, r.out_done[k], 0) == cudaSuccess;
        if (ok) {
            st = bf_gc_forward(p, d_in[k], d_out[k], ws, ws_bytes, (bf_stream_t)r.run);
            ok = st == BF_OK;
        }
        ok = ok && cudaEventRecord(r.run_done[k], r.run) == cudaSuccess;
        // download it
        ok = ok && cudaStreamWaitEvent(r.down, r.run_done[k], 0) == cudaSuccess &&
             cudaMemcpyAsync(h_out[i], d_out[k], bytes, cudaMemcpyDeviceToHost, r.down) == cudaSuccess &&
             cudaEventRecord(r.out_done[k], r.down) == cudaSuccess;
    }
    // wait for all three streams (also after a failure, so that no copy outlives the call)
    const bool synced = cudaStreamSynchronize(r.up) == cudaSuccess && cudaStreamSynchronize(r.run) == cudaSuccess &&
                        cudaStreamSynchronize(r.down) == cudaSuccess;
    if (st != BF_OK) return st;
    return ok && synced ? BF_OK : BF_ERR_CUDA;
}

}  // extern "C"
