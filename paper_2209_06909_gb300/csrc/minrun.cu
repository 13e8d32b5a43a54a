// minrun.cu -- Multiway Powersort with a minimum run length (Sec. 5, "Minimal
// run length"): a natural run shorter than m is extended to m elements (or to
// the end of the array) and sorted; the next run is searched from its end in
// the input as given.
//
// From a run start b the natural run is at least m long exactly when the m-1
// comparison flags lt[b+1 .. b+m-1] (lt[j]: a[j] < a[j-1]) are all equal; the
// run then ends at the end v of that stretch of equal flags, and otherwise at
// b + m.  A stretch of equal flags longer than one is the interior of one
// natural run [s, e) of the greedy partition (plus the flag at s when it
// continues the run's direction), so the natural runs with at least m-1
// interior flags give the "good intervals" [u-1, e-m+1) of start positions
// that take the natural run to e.  Between good intervals the starts advance
// by exactly m.  Position 0 and the end of every good interval are the nodes
// of a chain: from a node the progression c, c+m, ... continues until it
// lands in a good interval (the natural run ends at that interval's end, the
// next node) or reaches the end of the array.  Every node finds its successor
// on its own; pointer jumping then marks the chain that starts at position 0,
// a scan numbers its runs, and one pass writes them.
//
// Runs of at most m elements are sorted stably in a copy of the input, one
// thread each, by a sorting network on (key, position) pairs (any stable sort
// gives the same run; the paper extends runs with insertion sort); longer
// runs are natural runs, read forwards or (strictly descending) backwards by
// the merges.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

constexpr int kMrThreads = 256;
constexpr int kMrItems = 16;
constexpr uint32_t kMrTile = kMrThreads * kMrItems;

// Run [s, e) of the natural partition has at least m-1 interior flags: its
// start positions from u-1 to e-m take the natural run to e.  The flag at s
// belongs to the run's stretch when it has the run's direction (u = s), else
// u = s + 1; it matters only for a run of exactly m-1 elements (a longer run
// is good either way, a shorter one never), so the two keys at s are read
// only then, or when u itself is wanted.
template <typename K>
__device__ __forceinline__ uint32_t stretch_start(const K* __restrict__ keys, uint32_t s, uint32_t dir) {
    const uint32_t lt_s = s > 0 && keys[s] < keys[s - 1] ? 1u : 0u;
    return s + ((s > 0 && lt_s == dir) ? 0u : 1u);
}
template <typename K>
__device__ __forceinline__ bool good_run(const K* __restrict__ keys, uint32_t s, uint32_t e, uint32_t dir, uint32_t m) {
    const uint32_t len = e - s;
    if (len >= m) return true;
    if (len + 1 < m) return false;
    return stretch_start(keys, s, dir) == s;
}
// rs[i0 .. i0 + 16] (the run-start array is padded past r for 16-byte loads)
__device__ __forceinline__ void load_starts17(const uint32_t* __restrict__ rs, uint32_t i0, uint32_t (&v)[17]) {
    const uint4* r4 = reinterpret_cast<const uint4*>(rs + i0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint4 x = r4[q];
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
    v[16] = rs[i0 + 16];
}

// Per tile of kMrTile natural runs: the number of good runs.
template <typename K>
__global__ void __launch_bounds__(kMrThreads) k_mr_good_count(const uint64_t* __restrict__ ctr, const K* __restrict__ keys,
                                                             const uint32_t* __restrict__ rs,
                                                             const uint8_t* __restrict__ rdesc, uint32_t m,
                                                             uint32_t* __restrict__ tiles) {
    __shared__ uint32_t tmp[kMrThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t ntiles = (uint32_t)ceil_div(r, kMrTile);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = tile * kMrTile + threadIdx.x * kMrItems;
        uint32_t c = 0;
        if (i0 < r) {
            uint32_t v[17];
            load_starts17(rs, i0, v);
#pragma unroll
            for (uint32_t q = 0; q < (uint32_t)kMrItems; q++)
                if (i0 + q < r && good_run(keys, v[q], v[q + 1], rdesc[i0 + q], m)) c++;
        }
        uint32_t tot;
        block_sum_excl<kMrThreads>(c, tmp, &tot);
        if (threadIdx.x == 0) tiles[tile] = tot;
    }
}

// One block: exclusive scan of the per-tile counts of `count` items (count =
// *count_src + add, capped at item_cap), in place; the total goes to
// *total_dst.  A count beyond the capacities is reported.
__global__ void __launch_bounds__(1024) k_mr_scan_tiles(uint32_t* __restrict__ tiles, const uint64_t* __restrict__ count_src,
                                                       uint32_t add, uint32_t item_cap, uint64_t* __restrict__ total_dst,
                                                       uint32_t tiles_cap, uint32_t* __restrict__ status) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
    const uint64_t count = min(*count_src + add, (uint64_t)item_cap);
    const uint32_t ntiles = (uint32_t)ceil_div(count, kMrTile);
    if (ntiles > tiles_cap || *count_src + add > item_cap) {
        if (threadIdx.x == 0) dev_fail(status, kDevCapacity);
        if (ntiles > tiles_cap) return;
    }
    const uint32_t per = (ntiles + 1023) / 1024;
    const uint32_t b = min(ntiles, threadIdx.x * per), e = min(ntiles, b + per);
    uint32_t acc = 0;
    for (uint32_t t = b; t < e; t++) acc += tiles[t];
    uint32_t tot;
    uint32_t pre = block_sum_excl<1024>(acc, tmp, &tot);
    for (uint32_t t = b; t < e; t++) {
        const uint32_t c = tiles[t];
        tiles[t] = pre;
        pre += c;
    }
    if (threadIdx.x == 0) *total_dst = tot;
}

// Writes the good intervals in position order: gs = u - 1, ge = e - m + 1, gv = e.
template <typename K>
__global__ void __launch_bounds__(kMrThreads) k_mr_good_write(const uint64_t* __restrict__ ctr, const K* __restrict__ keys,
                                                             const uint32_t* __restrict__ rs,
                                                             const uint8_t* __restrict__ rdesc, uint32_t m,
                                                             const uint32_t* __restrict__ tiles, MinRunView mr) {
    __shared__ uint32_t tmp[kMrThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t ntiles = (uint32_t)ceil_div(r, kMrTile);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t i0 = tile * kMrTile + threadIdx.x * kMrItems;
        uint32_t flags = 0;
        uint32_t v[17];
        if (i0 < r) {
            load_starts17(rs, i0, v);
#pragma unroll
            for (uint32_t q = 0; q < (uint32_t)kMrItems; q++)
                if (i0 + q < r && good_run(keys, v[q], v[q + 1], rdesc[i0 + q], m)) flags |= 1u << q;
        }
        uint32_t at = tiles[tile] + block_sum_excl<kMrThreads>((uint32_t)__popc(flags), tmp, nullptr);
        while (flags) {
            const uint32_t q = __ffs(flags) - 1;
            flags &= flags - 1;
            const uint32_t sq = rs[i0 + q], e = rs[i0 + q + 1];
            const uint32_t u = stretch_start(keys, sq, (uint32_t)rdesc[i0 + q]);
            if (at < mr.cap) {
                mr.gs[at] = u - 1;
                mr.ge[at] = e - m + 1;
                mr.gv[at] = e;
            }
            at++;
        }
    }
}

// Successor of every node: node 0 is position 0, node j + 1 position gv[j].
// From c the starts are c, c + m, ...; the first good interval one of them
// lands in ends the progression with a natural run from that start h to the
// interval's end (node j + 1); without one the forced runs go on to the end
// of the array (the last start b has n - b <= m and takes all n - b elements).
__global__ void __launch_bounds__(kMrThreads) k_mr_succ(const uint64_t* __restrict__ ctr, uint64_t n, MinRunView mr) {
    const uint32_t R = min((uint32_t)ctr[kCtrMrGood], mr.cap);
    const uint32_t END = R + 1;
    const uint32_t m = mr.m;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x <= R + 1; x += gridDim.x * blockDim.x) {
        if (x == END) {
            mr.succ[x] = END;
            mr.hit[x] = (uint32_t)n;
            mr.cnt[x] = 0;
            continue;
        }
        const uint32_t c = x == 0 ? 0u : mr.gv[x - 1];
        uint32_t succ = END, hit = (uint32_t)n, cnt = 0;
        if (c < n) {
            uint32_t lo = 0, hi = R;  // first interval with ge > c
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (mr.ge[mid] > c) hi = mid; else lo = mid + 1;
            }
            for (uint32_t s = lo; s < R; s++) {
                const uint32_t g0 = max(mr.gs[s], c);
                const uint32_t h = c + (g0 - c + m - 1) / m * m;
                if (h < mr.ge[s]) {
                    succ = s + 1;
                    hit = h;
                    cnt = (h - c) / m + 1;
                    break;
                }
            }
            if (succ == END) cnt = (uint32_t)((n - c - 1) / m + 1);
        }
        mr.succ[x] = succ;
        mr.hit[x] = hit;
        mr.cnt[x] = cnt;
    }
}

__global__ void __launch_bounds__(kMrThreads) k_mr_jump_init(const uint64_t* __restrict__ ctr, MinRunView mr) {
    const uint32_t R = min((uint32_t)ctr[kCtrMrGood], mr.cap);
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x <= R + 1; x += gridDim.x * blockDim.x) {
        mr.mark[x] = x == 0 ? 1u : 0u;
        mr.jmp0[x] = mr.succ[x];
    }
}

// One round of pointer jumping: a marked node marks the node 2^t steps ahead,
// and the jump pointers double.  Marks only ever reach nodes on the chain from
// node 0, so a mark seen early within a round is harmless; after t rounds the
// first 2^t nodes of the chain are marked.
__global__ void __launch_bounds__(kMrThreads) k_mr_jump(const uint64_t* __restrict__ ctr, MinRunView mr,
                                                       const uint32_t* __restrict__ jin, uint32_t* __restrict__ jout) {
    const uint32_t R = min((uint32_t)ctr[kCtrMrGood], mr.cap);
    const uint32_t END = R + 1;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x <= END; x += gridDim.x * blockDim.x) {
        const uint32_t t = jin[x];
        if (t < END && mr.mark[x]) mr.mark[t] = 1u;
        jout[x] = t < END ? jin[t] : END;
    }
}

// Per tile of kMrTile nodes: the runs the marked nodes contribute.
__global__ void __launch_bounds__(kMrThreads) k_mr_node_sum(const uint64_t* __restrict__ ctr, MinRunView mr) {
    __shared__ uint32_t tmp[kMrThreads / 32 + 1];
    const uint32_t nodes = min((uint32_t)ctr[kCtrMrGood], mr.cap) + 1;
    const uint32_t ntiles = (uint32_t)ceil_div(nodes, kMrTile);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t x0 = tile * kMrTile + threadIdx.x * kMrItems;
        uint32_t c = 0;
        for (uint32_t q = 0; q < (uint32_t)kMrItems; q++)
            if (x0 + q < nodes && mr.mark[x0 + q]) c += mr.cnt[x0 + q];
        uint32_t tot;
        block_sum_excl<kMrThreads>(c, tmp, &tot);
        if (threadIdx.x == 0) mr.tiles[tile] = tot;
    }
}

// Index of each node's first run (exclusive prefix over marked nodes; an
// unmarked node contributes nothing and shares the next node's offset).
__global__ void __launch_bounds__(kMrThreads) k_mr_node_off(const uint64_t* __restrict__ ctr, MinRunView mr) {
    __shared__ uint32_t tmp[kMrThreads / 32 + 1];
    const uint32_t nodes = min((uint32_t)ctr[kCtrMrGood], mr.cap) + 1;
    const uint32_t ntiles = (uint32_t)ceil_div(nodes, kMrTile);
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t x0 = tile * kMrTile + threadIdx.x * kMrItems;
        uint32_t c = 0;
        for (uint32_t q = 0; q < (uint32_t)kMrItems; q++)
            if (x0 + q < nodes && mr.mark[x0 + q]) c += mr.cnt[x0 + q];
        uint32_t at = mr.tiles[tile] + block_sum_excl<kMrThreads>(c, tmp, nullptr);
        for (uint32_t q = 0; q < (uint32_t)kMrItems; q++) {
            if (x0 + q >= nodes) break;
            mr.off[x0 + q] = at;
            if (mr.mark[x0 + q]) at += mr.cnt[x0 + q];
        }
    }
}

// Run q of the partition: its start, the direction of its natural part
// (desc_nat, the tree output), and for the merges the direction of runs
// longer than m (shorter ones are sorted in the copy).
template <typename K>
__global__ void __launch_bounds__(kMrThreads) k_mr_write_runs(uint64_t* __restrict__ ctr, const K* __restrict__ keys,
                                                             uint64_t n, MinRunView mr, uint32_t* __restrict__ rs,
                                                             uint8_t* __restrict__ rdesc, uint32_t r_cap) {
    // every run but the last has at least two elements: r <= n/2 + 1 <= r_cap
    const uint32_t r = min((uint32_t)ctr[kCtrR], r_cap);
    const uint32_t nodes = min((uint32_t)ctr[kCtrMrGood], mr.cap) + 1;
    const uint32_t END = nodes;
    const uint32_t m = mr.m;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < r; q += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nodes - 1;  // last node with off <= q
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (mr.off[mid] <= q) lo = mid; else hi = mid - 1;
        }
        const uint32_t x = lo;
        const uint32_t j = q - mr.off[x];
        const uint32_t c = x == 0 ? 0u : mr.gv[x - 1];
        const bool hits = mr.succ[x] < END;
        const bool last = j + 1 == mr.cnt[x];
        uint32_t start, len;
        if (hits && last) {
            start = mr.hit[x];
            len = mr.gv[mr.succ[x] - 1] - start;
        } else {
            start = c + j * m;
            len = (hits || !last) ? m : (uint32_t)(n - start);
        }
        rs[q] = start;
        const uint8_t dir = (uint64_t)start + 1 < n && keys[start + 1] < keys[start] ? 1u : 0u;
        mr.desc_nat[q] = dir;
        rdesc[q] = (dir && len > m) ? 1u : 0u;
        if (q + 1 == r) rs[r] = (uint32_t)n;
    }
}

// (key, position) as one 64-bit word for 32-bit keys: comparing the words
// compares keys, then positions, so sorting them is a stable sort of the keys.
struct ShortItem32 {
    unsigned long long kp;
    __device__ __forceinline__ bool before(const ShortItem32& o) const { return kp < o.kp; }
};
struct ShortItem64 {
    uint64_t key;
    uint32_t pos;
    __device__ __forceinline__ bool before(const ShortItem64& o) const {
        return key < o.key || (key == o.key && pos < o.pos);
    }
};

template <typename T>
__device__ __forceinline__ void cswap(T& a, T& b, uint32_t& va, uint32_t& vb) {
    const bool sw = b.before(a);
    const T lo = sw ? b : a, hi = sw ? a : b;
    const uint32_t vlo = sw ? vb : va, vhi = sw ? va : vb;
    a = lo;
    b = hi;
    va = vlo;
    vb = vhi;
}

// Batcher's odd-even merge sort network on 32 inputs: 191 compare-exchanges
// (i, j), i < j, in order (table below).
constexpr int kNet32Len = 191;

// The network on 32 items held in registers: the loop is unrolled, so every
// index is a compile-time constant.
template <typename F>
__device__ __forceinline__ void for_net32(F&& cas) {
    constexpr uint8_t net[kNet32Len][2] = {
    {0, 1}, {2, 3}, {4, 5}, {6, 7}, {8, 9}, {10, 11}, {12, 13}, {14, 15}, {16, 17}, {18, 19}, {20, 21}, {22, 23},
    {24, 25}, {26, 27}, {28, 29}, {30, 31}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {8, 10}, {9, 11}, {12, 14}, {13, 15},
    {16, 18}, {17, 19}, {20, 22}, {21, 23}, {24, 26}, {25, 27}, {28, 30}, {29, 31}, {1, 2}, {5, 6}, {9, 10}, {13, 14},
    {17, 18}, {21, 22}, {25, 26}, {29, 30}, {0, 4}, {1, 5}, {2, 6}, {3, 7}, {8, 12}, {9, 13}, {10, 14}, {11, 15},
    {16, 20}, {17, 21}, {18, 22}, {19, 23}, {24, 28}, {25, 29}, {26, 30}, {27, 31}, {2, 4}, {3, 5}, {10, 12}, {11, 13},
    {18, 20}, {19, 21}, {26, 28}, {27, 29}, {1, 2}, {3, 4}, {5, 6}, {9, 10}, {11, 12}, {13, 14}, {17, 18}, {19, 20},
    {21, 22}, {25, 26}, {27, 28}, {29, 30}, {0, 8}, {1, 9}, {2, 10}, {3, 11}, {4, 12}, {5, 13}, {6, 14}, {7, 15},
    {16, 24}, {17, 25}, {18, 26}, {19, 27}, {20, 28}, {21, 29}, {22, 30}, {23, 31}, {4, 8}, {5, 9}, {6, 10}, {7, 11},
    {20, 24}, {21, 25}, {22, 26}, {23, 27}, {2, 4}, {3, 5}, {6, 8}, {7, 9}, {10, 12}, {11, 13}, {18, 20}, {19, 21},
    {22, 24}, {23, 25}, {26, 28}, {27, 29}, {1, 2}, {3, 4}, {5, 6}, {7, 8}, {9, 10}, {11, 12}, {13, 14}, {17, 18},
    {19, 20}, {21, 22}, {23, 24}, {25, 26}, {27, 28}, {29, 30}, {0, 16}, {1, 17}, {2, 18}, {3, 19}, {4, 20}, {5, 21},
    {6, 22}, {7, 23}, {8, 24}, {9, 25}, {10, 26}, {11, 27}, {12, 28}, {13, 29}, {14, 30}, {15, 31}, {8, 16}, {9, 17},
    {10, 18}, {11, 19}, {12, 20}, {13, 21}, {14, 22}, {15, 23}, {4, 8}, {5, 9}, {6, 10}, {7, 11}, {12, 16}, {13, 17},
    {14, 18}, {15, 19}, {20, 24}, {21, 25}, {22, 26}, {23, 27}, {2, 4}, {3, 5}, {6, 8}, {7, 9}, {10, 12}, {11, 13},
    {14, 16}, {15, 17}, {18, 20}, {19, 21}, {22, 24}, {23, 25}, {26, 28}, {27, 29}, {1, 2}, {3, 4}, {5, 6}, {7, 8},
    {9, 10}, {11, 12}, {13, 14}, {15, 16}, {17, 18}, {19, 20}, {21, 22}, {23, 24}, {25, 26}, {27, 28}, {29, 30},
    };
#pragma unroll
    for (int c = 0; c < kNet32Len; c++) cas(net[c][0], net[c][1]);
}

template <typename T>
__device__ __forceinline__ void sort_net32(T (&x)[32], uint32_t (&v)[32]) {
    for_net32([&](int i, int j) { cswap(x[i], x[j], v[i], v[j]); });
}

// Keys alone: equal keys cannot be told apart, so the plain network (min and
// max per pair) gives the stable sort's output.
template <typename K>
__device__ __forceinline__ void sort_net32_keys(K (&x)[32]) {
    for_net32([&](int i, int j) {
        const K a = x[i], b = x[j];
        x[i] = a < b ? a : b;
        x[j] = a < b ? b : a;
    });
}

// Elements of the runs of one warp staged in shared memory: at most 32 runs of
// at most 32 elements, with one pad slot after every 32 (so that lanes whose
// runs start a multiple of 8 apart still read different banks).
constexpr uint32_t kMrWarpSpan = 32 * 32;
constexpr uint32_t kMrWarpSlots = kMrWarpSpan + kMrWarpSpan / 32;
__device__ __forceinline__ uint32_t mr_slot(uint32_t j) { return j + (j >> 5); }

template <typename K, bool V>
struct MrSortSmem {
    static constexpr size_t bytes() { return (size_t)(kMrThreads / 32) * kMrWarpSlots * (sizeof(K) + (V ? 4 : 0)); }
};

// One thread per run of at most m <= 32 elements: the run is loaded into
// registers (padded with items that sort last), sorted (with payloads: stably
// by (key, position); keys alone by key), and rewritten in place in the copy.
// A warp takes 32 consecutive
// runs; when they span at most kMrWarpSpan elements (every run short, as in a
// permutation) the warp stages the span in shared memory with coalesced loads
// and stores it back the same way, else each thread reads and writes its run
// in global memory directly.
template <typename K, bool V>
__global__ void __launch_bounds__(kMrThreads, V ? 1 : 2) k_mr_sort_short(const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs,
                                                             uint32_t m, K* __restrict__ copy, uint32_t* __restrict__ vcopy,
                                                             uint32_t r_cap) {
    using T = typename std::conditional<sizeof(K) == 4, ShortItem32, ShortItem64>::type;
    extern __shared__ uint4 mr_smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    K* wk = reinterpret_cast<K*>(mr_smem) + (size_t)warp * kMrWarpSlots;
    uint32_t* wv = V ? reinterpret_cast<uint32_t*>(reinterpret_cast<K*>(mr_smem) + (size_t)(kMrThreads / 32) * kMrWarpSlots) +
                           (size_t)warp * kMrWarpSlots
                     : nullptr;
    const uint32_t r = min((uint32_t)ctr[kCtrR], r_cap);
    const uint32_t warps = gridDim.x * (kMrThreads / 32);
    for (uint32_t g0 = (blockIdx.x * (kMrThreads / 32) + warp) * 32u; g0 < r; g0 += warps * 32u) {
        const uint32_t q = g0 + lane;
        const uint32_t s = q < r ? rs[q] : 0u;
        const uint32_t e = q < r ? rs[q + 1] : 0u;
        const uint32_t len = e - s;
        const bool mine = q < r && len >= 2 && len <= m;
        const uint32_t S = __shfl_sync(0xffffffffu, s, 0);
        const uint32_t last = min(32u, r - g0) - 1u;
        const uint32_t E = __shfl_sync(0xffffffffu, e, last);
        const bool staged = E - S <= kMrWarpSpan;  // the same for the whole warp
        if (staged) {
            for (uint32_t i = lane; i < E - S; i += 32) {
                wk[mr_slot(i)] = copy[S + i];
                if (V) wv[mr_slot(i)] = vcopy[S + i];
            }
            __syncwarp();
        }
        if (!V && mine) {
            const uint32_t b = s - S;
            K xk[32];
#pragma unroll
            for (uint32_t i = 0; i < 32; i++) xk[i] = i < len ? (staged ? wk[mr_slot(b + i)] : copy[s + i]) : ~K(0);
            sort_net32_keys(xk);
#pragma unroll
            for (uint32_t i = 0; i < 32; i++) {
                if (i < len) {
                    if (staged) wk[mr_slot(b + i)] = xk[i];
                    else copy[s + i] = xk[i];
                }
            }
        }
        if (V && mine) {
            const uint32_t b = s - S;
            T x[32];
            uint32_t v[32];
#pragma unroll
            for (uint32_t i = 0; i < 32; i++) {
                const bool in = i < len;
                const K key = in ? (staged ? wk[mr_slot(b + i)] : copy[s + i]) : ~K(0);
                if constexpr (sizeof(K) == 4) {
                    x[i].kp = ((unsigned long long)key << 32) | (in ? i : 32u + i);
                } else {
                    x[i].key = key;
                    x[i].pos = in ? i : 32u + i;
                }
                v[i] = (V && in) ? (staged ? wv[mr_slot(b + i)] : vcopy[s + i]) : 0u;
            }
            sort_net32(x, v);
#pragma unroll
            for (uint32_t i = 0; i < 32; i++) {
                if (i < len) {
                    K key;
                    if constexpr (sizeof(K) == 4) key = (K)(x[i].kp >> 32);
                    else key = x[i].key;
                    if (staged) {
                        wk[mr_slot(b + i)] = key;
                        if (V) wv[mr_slot(b + i)] = v[i];
                    } else {
                        copy[s + i] = key;
                        if (V) vcopy[s + i] = v[i];
                    }
                }
            }
        }
        if (staged) {
            __syncwarp();
            for (uint32_t i = lane; i < E - S; i += 32) {
                copy[S + i] = wk[mr_slot(i)];
                if (V) vcopy[S + i] = wv[mr_slot(i)];
            }
            __syncwarp();
        }
    }
}

}  // namespace

// ----------------------------------------------------------------- launcher

template <typename K, bool V>
void launch_min_run(const K* keys, K* copy, uint32_t* vcopy, uint64_t n, const MinRunView& mr, const WsView& ws,
                    cudaStream_t st) {
    const uint32_t r_bound = (uint32_t)std::min<uint64_t>(n / 2 + 2, n + 1);
    const uint32_t grid_tiles = (uint32_t)std::min<uint64_t>(ceil_div(r_bound, kMrTile), 152 * 8);
    uint32_t* status = reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus);
    // good intervals from the natural partition
    k_mr_good_count<K><<<grid_tiles, kMrThreads, 0, st>>>(ws.counters, keys, ws.run_starts, ws.run_desc, mr.m, mr.tiles);
    k_mr_scan_tiles<<<1, 1024, 0, st>>>(mr.tiles, ws.counters + kCtrR, 0u, r_bound, ws.counters + kCtrMrGood, mr.tiles_cap,
                                        status);
    k_mr_good_write<K><<<grid_tiles, kMrThreads, 0, st>>>(ws.counters, keys, ws.run_starts, ws.run_desc, mr.m, mr.tiles, mr);
    // the chain from position 0
    const uint32_t node_grid = (uint32_t)std::min<uint64_t>(ceil_div((uint64_t)mr.cap + 2, kMrThreads), 152 * 16);
    k_mr_succ<<<node_grid, kMrThreads, 0, st>>>(ws.counters, n, mr);
    k_mr_jump_init<<<node_grid, kMrThreads, 0, st>>>(ws.counters, mr);
    int rounds = 0;
    while ((1ull << rounds) < (uint64_t)mr.cap + 2) rounds++;
    for (int t = 0; t < rounds; t++) {
        const uint32_t* jin = (t & 1) ? mr.jmp1 : mr.jmp0;
        uint32_t* jout = (t & 1) ? mr.jmp0 : mr.jmp1;
        k_mr_jump<<<node_grid, kMrThreads, 0, st>>>(ws.counters, mr, jin, jout);
    }
    // runs of the chain, numbered in order
    const uint32_t node_tiles = (uint32_t)std::min<uint64_t>(ceil_div((uint64_t)mr.cap + 1, kMrTile), 152 * 8);
    k_mr_node_sum<<<node_tiles, kMrThreads, 0, st>>>(ws.counters, mr);
    // nodes: position 0 and the end of every good interval (at most cap of them)
    k_mr_scan_tiles<<<1, 1024, 0, st>>>(mr.tiles, ws.counters + kCtrMrGood, 1u, mr.cap + 1, ws.counters + kCtrR,
                                        mr.tiles_cap, status);
    k_mr_node_off<<<node_tiles, kMrThreads, 0, st>>>(ws.counters, mr);
    const uint32_t run_grid = (uint32_t)std::min<uint64_t>(ceil_div(r_bound, kMrThreads), 152 * 16);
    k_mr_write_runs<K><<<run_grid, kMrThreads, 0, st>>>(ws.counters, keys, n, mr, ws.run_starts, ws.run_desc, r_bound);
    // the copy: every run of at most m elements sorted in place
    const size_t sort_smem = MrSortSmem<K, V>::bytes();
    cudaFuncSetAttribute(k_mr_sort_short<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
    k_mr_sort_short<K, V><<<(uint32_t)std::min<uint64_t>(ceil_div((uint64_t)r_bound, kMrThreads), 152 * 16), kMrThreads,
                            sort_smem, st>>>(ws.counters, ws.run_starts, mr.m, copy, vcopy, r_bound);
    g_launches += 9 + rounds;
}

#define MPS_INST(K, V) \
    template void launch_min_run<K, V>(const K*, K*, uint32_t*, uint64_t, const MinRunView&, const WsView&, cudaStream_t);
MPS_INST(uint32_t, false)
MPS_INST(uint32_t, true)
MPS_INST(uint64_t, false)
MPS_INST(uint64_t, true)
#undef MPS_INST

}  // namespace mps
