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
// Runs of at most m elements are sorted stably by one warp each (rank of every
// element under (key, position)) in a copy of the input; longer runs are
// natural runs, read forwards or (strictly descending) backwards by the merges.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

constexpr int kMrThreads = 256;
constexpr int kMrItems = 16;
constexpr uint32_t kMrTile = kMrThreads * kMrItems;

// Run i of the natural partition has at least m-1 interior flags: its start
// positions from u-1 to e-m take the natural run to e.
template <typename K>
__device__ __forceinline__ bool good_run(const K* __restrict__ keys, const uint32_t* __restrict__ rs,
                                         const uint8_t* __restrict__ rdesc, uint32_t i, uint32_t m, uint32_t* u_out,
                                         uint32_t* e_out) {
    const uint32_t s = rs[i], e = rs[i + 1];
    const uint32_t dir = rdesc[i];
    // the flag at s belongs to the stretch when it has the run's direction
    const uint32_t lt_s = s > 0 && keys[s] < keys[s - 1] ? 1u : 0u;
    const uint32_t u = s + ((s > 0 && lt_s == dir) ? 0u : 1u);
    *u_out = u;
    *e_out = e;
    return e >= u && e - u + 1 >= m;
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
        for (uint32_t q = 0; q < (uint32_t)kMrItems; q++) {
            uint32_t u, e;
            if (i0 + q < r && good_run(keys, rs, rdesc, i0 + q, m, &u, &e)) c++;
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
        for (uint32_t q = 0; q < (uint32_t)kMrItems; q++) {
            uint32_t u, e;
            if (i0 + q < r && good_run(keys, rs, rdesc, i0 + q, m, &u, &e)) flags |= 1u << q;
        }
        uint32_t at = tiles[tile] + block_sum_excl<kMrThreads>((uint32_t)__popc(flags), tmp, nullptr);
        while (flags) {
            const uint32_t q = __ffs(flags) - 1;
            flags &= flags - 1;
            uint32_t u, e;
            good_run(keys, rs, rdesc, i0 + q, m, &u, &e);
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

// One warp per run of at most m <= 32 elements: every element's rank under
// (key, position), i.e. its place in the stable sort of the run; the run is
// rewritten in place in the copy.
template <typename K, bool V>
__global__ void __launch_bounds__(kMrThreads) k_mr_sort_short(const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs,
                                                             uint32_t m, K* __restrict__ copy, uint32_t* __restrict__ vcopy,
                                                             uint32_t r_cap) {
    const uint32_t r = min((uint32_t)ctr[kCtrR], r_cap);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = warp; q < r; q += nwarps) {
        const uint32_t s = rs[q], len = rs[q + 1] - s;
        if (len > m || len < 2) continue;
        const K key = lane < len ? copy[s + lane] : K(0);
        const uint32_t val = (V && lane < len) ? vcopy[s + lane] : 0u;
        uint32_t rank = 0;
        for (uint32_t t = 0; t < len; t++) {
            const K kt = __shfl_sync(0xffffffffu, key, t);
            rank += (kt < key || (kt == key && t < lane)) ? 1u : 0u;
        }
        __syncwarp();
        if (lane < len) {
            copy[s + rank] = key;
            if (V) vcopy[s + rank] = val;
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
    k_mr_sort_short<K, V><<<(uint32_t)std::min<uint64_t>(ceil_div((uint64_t)r_bound * 32, kMrThreads), 152 * 32), kMrThreads, 0,
                            st>>>(ws.counters, ws.run_starts, mr.m, copy, vcopy, r_bound);
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
