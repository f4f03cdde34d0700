// bf_gc_forward_static: the forward filter with its scratch in a file-scope device array,
// for callers that cannot allocate device memory when they filter.  Nothing in the
// paper corresponds to this; it only changes where the workspace lives.
#include <mutex>

#include "bfgc_internal.h"

// One scratch area per device that loads the library, alive until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[BF_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device with
// that device current and cached.
bf_status static_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return BF_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_gc_forward_static(bf_gc_plan_t plan, const float* d_f, float* d_out,
                                          bf_stream_t stream) {
    if (!plan || !d_f || !d_out) return BF_ERR_INVALID_ARG;
    size_t need = 0;
    bf_status st = bf_gc_workspace_size(plan, &need, nullptr);
    if (st != BF_OK) return st;
    if (need > (size_t)BF_STATIC_SCRATCH_BYTES) return BF_ERR_WORKSPACE;
    void* ws = nullptr;
    if ((st = static_scratch(&ws)) != BF_OK) return st;
    return bf_gc_forward(plan, d_f, d_out, ws, (size_t)BF_STATIC_SCRATCH_BYTES, stream);
}
