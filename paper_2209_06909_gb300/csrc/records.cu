// records.cu -- stable sort of records: a key and a 64-bit payload (Sec. 5,
// "records" experiment: a long key and a pointer, 16 bytes).
//
// The payloads are not carried through the merge levels.  The keys are sorted
// with a uint32 payload holding each record's input index (mps_sort_pairs,
// stable), which yields the stable permutation; one gather then moves every
// 64-bit payload once, out[i] = in[perm[i]].  The result equals carrying the
// payloads through every merge, since the index order is the stable order.
#include <algorithm>
#include <cstdint>

#include "../../include/mps.h"
#include "common.cuh"

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

__global__ void __launch_bounds__(256) k_iota(uint32_t* __restrict__ idx, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        idx[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(256) k_gather_u64(const uint64_t* __restrict__ in, const uint32_t* __restrict__ perm,
                                                   uint64_t* __restrict__ out, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(b);
    return na && nb && x < y + nb && y < x + na;
}

}  // namespace

extern "C" {

mps_status mps_records_workspace_size(uint64_t n, mps_key_type kt, int k, size_t* bytes) {
    if (!bytes) return MPS_ERR_INVALID_ARG;
    size_t pairs = 0;
    const mps_status s = mps_workspace_size(n, kt, 1, k, &pairs);
    if (s != MPS_OK) return s;
    *bytes = align_up(pairs) + 2 * align_up((size_t)std::max<uint64_t>(n, 1) * 4);
    return MPS_OK;
}

mps_status mps_sort_records(const void* d_keys_in, const uint64_t* d_vals_in, void* d_keys_out, uint64_t* d_vals_out,
                            uint64_t n, mps_key_type kt, int k, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    size_t need = 0;
    mps_status s = mps_records_workspace_size(n, kt, k, &need);
    if (s != MPS_OK) return s;
    if (n == 0) return MPS_OK;
    if (!d_keys_in || !d_vals_in || !d_keys_out || !d_vals_out || !d_ws) return MPS_ERR_INVALID_ARG;
    if (ws_bytes < need) return MPS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(d_ws) % 16) return MPS_ERR_INVALID_ARG;
    if (overlaps(d_vals_in, n * 8, d_vals_out, n * 8)) return MPS_ERR_INVALID_ARG;
    size_t pairs = 0;
    mps_workspace_size(n, kt, 1, k, &pairs);
    char* w = static_cast<char*>(d_ws);
    uint32_t* idx = reinterpret_cast<uint32_t*>(w + align_up(pairs));
    uint32_t* perm = reinterpret_cast<uint32_t*>(w + align_up(pairs) + align_up(n * 4));
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 152 * 8);
    k_iota<<<grid, 256, 0, stream>>>(idx, n);
    if (cudaGetLastError() != cudaSuccess) return MPS_ERR_CUDA;
    s = mps_sort_pairs(d_keys_in, idx, d_keys_out, perm, n, kt, k, d_ws, pairs, nullptr, stream);
    if (s != MPS_OK) return s;
    k_gather_u64<<<grid, 256, 0, stream>>>(d_vals_in, perm, d_vals_out, n);
    if (cudaGetLastError() != cudaSuccess) return MPS_ERR_CUDA;
    return MPS_OK;
}

}  // extern "C"
