// common.cuh -- shared device utilities of the CUDA path (block scans, shuffles,
// status word).  Nothing here is shared with the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mps {

constexpr uint32_t kNone = 0xFFFFFFFFu;

// Device-side error codes written to the status word (first error wins).
enum DevError : uint32_t {
    kDevOk = 0,
    kDevDegree = 1,      // a node had more than k-1 equal-power boundaries
    kDevCapacity = 2,    // a per-call capacity bound was exceeded
    kDevRange = 3,       // a tile did not fit its shared-memory capacity
    kDevUnitNode = 11,   // a work-unit interval pointed outside its level's nodes
    kDevUnitRange = 12,  // a work unit's slices or output left the key range
    kDevFusedRange = 13, // a fused subtree left the key range
    kDevLoneRange = 14,  // a lone run left the key range
    kDevPackNode = 15,   // packing saw an interval outside its level's nodes
    kDevMaxLen = 16,     // a batch array was longer than the caller's max_len
    kDevSpin = 17,       // a bounded wait on another block ran out
    kDevSplitSlot = 18,  // a splitter ranked outside its node's splitters (children not sorted)
    kDevLevelBound = 19, // a node larger than a fused tile at a power above the host's level bound
    kDevTail = 20,       // final-collapse variant: too many stack boundaries, or relabelled powers above 32
};

__device__ __forceinline__ void dev_fail(uint32_t* status, uint32_t code) { atomicCAS(status, 0u, code); }

// ---------------------------------------------------------------- shuffles
__device__ __forceinline__ uint32_t shfl_up(uint32_t v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint32_t shfl_down(uint32_t v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ unsigned long long shfl_up(unsigned long long v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ unsigned long long shfl_down(unsigned long long v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ uint4 shfl_up(uint4 v, int o) {
    v.x = __shfl_up_sync(0xffffffffu, v.x, o); v.y = __shfl_up_sync(0xffffffffu, v.y, o);
    v.z = __shfl_up_sync(0xffffffffu, v.z, o); v.w = __shfl_up_sync(0xffffffffu, v.w, o);
    return v;
}
__device__ __forceinline__ uint4 shfl_down(uint4 v, int o) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, o); v.y = __shfl_down_sync(0xffffffffu, v.y, o);
    v.z = __shfl_down_sync(0xffffffffu, v.z, o); v.w = __shfl_down_sync(0xffffffffu, v.w, o);
    return v;
}

// ------------------------------------------------------------ block scans
// Exclusive scan of one value per thread in thread order (REV = false) or in
// reverse thread order (REV = true, i.e. a suffix scan).  `op(a, b)` combines
// a segment a with the segment b that follows it in scan order.  `tmp` holds
// NT/32 + 1 entries of shared memory.  Returns the exclusive prefix; *total
// receives the aggregate of all threads.  Contains __syncthreads().
template <class T> struct NoDeduce { using type = T; };

template <int NT, bool REV, typename T, typename Op>
__device__ __forceinline__ T block_scan_excl(T v, Op op, typename NoDeduce<T>::type identity, T* tmp,
                                             typename NoDeduce<T>::type* total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpos = REV ? (NW - 1 - warp) : warp;   // warp position in scan order
    const int lpos = REV ? (31 - lane) : lane;       // lane position in scan order
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = REV ? shfl_down(x, o) : shfl_up(x, o);
        if (lpos >= o) x = op(y, x);
    }
    if (lpos == 31) tmp[wpos] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? tmp[lane] : identity;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = shfl_up(w, o);
            if (lane >= o && lane < NW) w = op(y, w);
        }
        if (lane < NW) tmp[lane] = w;
    }
    __syncthreads();
    T in_warp = REV ? shfl_down(x, 1) : shfl_up(x, 1);
    T pre = wpos > 0 ? tmp[wpos - 1] : identity;
    T res = lpos > 0 ? op(pre, in_warp) : pre;
    if (total) *total = tmp[NW - 1];
    __syncthreads();
    return res;
}

struct OpAdd32 { __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; } };
struct OpAddU64 {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a + b; }
};
struct OpOrU64 {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a | b; }
};
struct OpMax32 { __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; } };

template <int NT>
__device__ __forceinline__ uint32_t block_sum_excl(uint32_t v, uint32_t* tmp, uint32_t* total) {
    return block_scan_excl<NT, false>(v, OpAdd32(), 0u, tmp, total);
}

// Block-wide reductions (result valid in every thread).
template <int NT, typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, typename NoDeduce<T>::type identity, T* tmp) {
    T total;
    block_scan_excl<NT, false>(v, op, identity, tmp, &total);
    return total;
}

// ----------------------------------------------------------------- keys
template <typename K> struct KeyTraits;
template <> struct KeyTraits<uint32_t> { static constexpr int kBytes = 4; };
template <> struct KeyTraits<uint64_t> { static constexpr int kBytes = 8; };

__host__ __device__ constexpr uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

}  // namespace mps
