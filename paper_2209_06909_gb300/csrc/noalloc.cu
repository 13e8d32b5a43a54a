// noalloc.cu -- a sort entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a sort: code that
// runs inside a memory pool it does not own, plugin hosts that forbid device
// allocations after start-up, or real-time paths where an allocation (and the
// implicit device synchronisation it may cause) is not allowed.  For them,
// mps_sort_keys_noalloc sorts up to kNoAllocMaxN keys using a fixed scratch
// area that lives in the library itself: a file-scope __device__ array of
// kNoAllocScratchBytes bytes.  Every GPU that loads the library holds this
// array until the process exits.
//
// The array's name, used in host code, is only a host-side stand-in for the
// symbol: it is not a device address.  The device address is obtained once
// per device with cudaGetSymbolAddress (with that device current) and then
// handed to the regular sort as its workspace.
#include <cstdint>
#include <mutex>

#include "../../include/mps.h"

namespace {

constexpr uint64_t kNoAllocMaxN = 1ull << 20;                 // keys per call
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;     // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Looks up (once per device, with that device current) the device address of
// the scratch array.
mps_status scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MPS_ERR_CUDA;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return MPS_OK;
}

}  // namespace

extern "C" mps_status mps_sort_keys_noalloc(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt,
                                            int k, cudaStream_t stream) {
    if (n > kNoAllocMaxN) return MPS_ERR_WORKSPACE;
    size_t need = 0;
    mps_status s = mps_workspace_size(n, kt, 0, k, &need);
    if (s != MPS_OK) return s;
    if (need > kNoAllocScratchBytes) return MPS_ERR_WORKSPACE;
    void* scratch = nullptr;
    s = scratch_for_current_device(&scratch);
    if (s != MPS_OK) return s;
    // The sort clears the scratch it needs zeroed (its counter block) at the
    // start of every call, so what a previous call left behind is harmless.
    return mps_sort_keys(d_keys_in, d_keys_out, n, kt, k, scratch, kNoAllocScratchBytes, nullptr, stream);
}
