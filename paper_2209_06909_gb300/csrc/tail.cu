// tail.cu -- Alg. 2's final collapse by count instead of by power.
//
// After the last run, Alg. 2's stack holds the segments whose right-end
// boundary b has P_b <= P_c for every later boundary c: nothing after b had a
// smaller power, so nothing merged them.  Their powers never decrease up the
// stack.  The power rule (Alg. 1's tree, which the rest of the library
// builds) empties the stack in groups of equal power.  Two other ways appear
// in the paper:
//   policy 1: Alg. 2's last loop as printed pops up to k-1 entries per merge;
//   policy 2: the appendix's merge_down (k = 4, taken to any k) first pops
//             x = (entries mod (k-1)) entries, then k-1 at a time.
// Either way the final collapse is a chain of nodes over consecutive groups
// of stack boundaries: the rightmost group merges first (with the last run),
// the leftmost group last (the root).
//
// The library executes the tree whose nodes are the groups of equal power
// between nearest smaller powers.  The chain is that tree for these labels:
// a boundary left on the stack gets the number of its group counted from the
// left (1 .. m for m groups); every other boundary gets its power plus m.  A
// segment on the stack contains only boundaries of power above its right-end
// boundary's (they were merged before it was pushed), so after the shift they
// lie above every label of the chain, and the subtrees below the chain keep
// their shape (a common shift keeps the order of powers).  Every later kernel
// (min-tree, depths and merge cost, node table, fused and level merges) runs
// unchanged on the relabelled powers.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

constexpr int kTailThreads = 256;
constexpr int kTailItems = kMaskTile / kTailThreads;
static_assert(kTailItems == 16, "one 16-byte word of powers per thread");

struct OpMinU32 {
    __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a < b ? a : b; }
};

// Tiles of kMaskTile boundary slots covering boundaries 0..r.
__device__ __forceinline__ uint32_t tail_tiles(uint32_t r) { return (uint32_t)ceil_div((uint64_t)r + 1, kMaskTile); }

// The 16 powers of slots b0 .. b0+15 (b0 a multiple of 16, b0 <= r; the array
// is padded with 255 to a multiple of 32 slots past r, so the word is inside).
__device__ __forceinline__ uint4 load_word(const uint8_t* powers, uint32_t b0) {
    return *reinterpret_cast<const uint4*>(powers + b0);
}
__device__ __forceinline__ uint32_t byte_of(const uint4& w, int q) {
    const uint32_t x = q < 4 ? w.x : (q < 8 ? w.y : (q < 12 ? w.z : w.w));
    return (x >> (8 * (q & 3))) & 0xFFu;
}
__device__ __forceinline__ void set_byte(uint4& w, int q, uint32_t v) {
    uint32_t* x = q < 4 ? &w.x : (q < 8 ? &w.y : (q < 12 ? &w.z : &w.w));
    const uint32_t sh = 8 * (q & 3);
    *x = (*x & ~(0xFFu << sh)) | ((v & 0xFFu) << sh);
}

// Smallest power of the boundaries 1..r-1 in each tile (255 for none).
__global__ void __launch_bounds__(kTailThreads) k_tail_tilemin(const uint8_t* __restrict__ powers, const uint64_t* __restrict__ ctr,
                                                              unsigned long long* __restrict__ tmin) {
    __shared__ uint32_t tmp[kTailThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t tiles = tail_tiles(r);
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t b0 = tile * kMaskTile + threadIdx.x * kTailItems;
        uint32_t m = 255u;
        if (b0 <= r) {
            const uint4 w = load_word(powers, b0);
#pragma unroll
            for (int q = 0; q < kTailItems; q++) {
                const uint32_t b = b0 + q;
                if (b >= 1 && b < r) m = min(m, byte_of(w, q));
            }
        }
        m = block_reduce<kTailThreads>(m, OpMinU32(), 255u, tmp);
        if (threadIdx.x == 0) tmin[tile] = m;
    }
}

// tsuf[t] = smallest power in the tiles after t (255 for none).  One block.
__global__ void __launch_bounds__(1024) k_tail_tilescan(const uint64_t* __restrict__ ctr, const unsigned long long* __restrict__ tmin,
                                                        unsigned long long* __restrict__ tsuf) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
    const uint32_t tiles = tail_tiles((uint32_t)ctr[kCtrR]);
    const uint32_t per = (tiles + 1023) / 1024;
    const uint32_t t0 = min(tiles, threadIdx.x * per), t1 = min(tiles, t0 + per);
    uint32_t mine = 255u;
    for (uint32_t t = t0; t < t1; t++) mine = min(mine, (uint32_t)tmin[t]);
    uint32_t acc = block_scan_excl<1024, true>(mine, OpMinU32(), 255u, tmp, nullptr);  // tiles of later threads
    for (uint32_t t = t1; t > t0; t--) {
        tsuf[t - 1] = acc;
        acc = min(acc, (uint32_t)tmin[t - 1]);
    }
}

// Marks the boundaries left on the stack (P_b <= every later power): lists
// them, sets bit 7 of their power byte, and copies the original powers 0..r
// to orig (if given).
__global__ void __launch_bounds__(kTailThreads) k_tail_mark(uint8_t* __restrict__ powers, uint64_t* __restrict__ ctr,
                                                           const unsigned long long* __restrict__ tsuf,
                                                           uint32_t* __restrict__ list, uint8_t* __restrict__ orig) {
    __shared__ uint32_t tmp[kTailThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t tiles = tail_tiles(r);
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t b0 = tile * kMaskTile + threadIdx.x * kTailItems;
        const bool live = b0 <= r;
        uint4 w = make_uint4(~0u, ~0u, ~0u, ~0u);
        if (live) w = load_word(powers, b0);
        uint32_t mine = 255u;
#pragma unroll
        for (int q = 0; q < kTailItems; q++) {
            const uint32_t b = b0 + q;
            if (b >= 1 && b < r) mine = min(mine, byte_of(w, q));
        }
        // smallest power after this thread's slots: later threads of the tile, then later tiles
        uint32_t later = block_scan_excl<kTailThreads, true>(mine, OpMinU32(), 255u, tmp, nullptr);
        later = min(later, (uint32_t)tsuf[tile]);
        if (live) {
            if (orig)
                for (int q = 0; q < kTailItems && b0 + q <= r; q++) orig[b0 + q] = (uint8_t)byte_of(w, q);
            uint4 nw = w;
            bool changed = false;
            for (int q = kTailItems - 1; q >= 0; q--) {
                const uint32_t b = b0 + q;
                if (b < 1 || b >= r) continue;
                const uint32_t p = byte_of(w, q);
                if (p <= later) {
                    const uint32_t slot = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrTailCount), 1ull);
                    if (slot < kTailCap) list[slot] = b;
                    set_byte(nw, q, p | 0x80u);
                    changed = true;
                }
                later = min(later, p);
            }
            if (changed) *reinterpret_cast<uint4*>(powers + b0) = nw;
        }
    }
}

// One block of kTailCap threads: orders the s listed boundaries, groups them
// from the right by the policy, and writes label | 0x80 into their power
// bytes (label = group number counted from the left, 1 .. m).  Sets
// ctr[kCtrTailShift] = m and clears the power bit set (rebuilt by the apply).
__global__ void __launch_bounds__(kTailCap) k_tail_assign(uint8_t* __restrict__ powers, uint64_t* __restrict__ ctr,
                                                         const uint32_t* __restrict__ list, int k, int policy) {
    __shared__ uint32_t sl[kTailCap];
    uint32_t* status = reinterpret_cast<uint32_t*>(ctr + kCtrStatus);
    const uint64_t cnt = ctr[kCtrTailCount];
    if (cnt > kTailCap) {
        if (threadIdx.x == 0) {
            dev_fail(status, kDevTail);
            ctr[kCtrTailShift] = 0;
        }
        return;
    }
    const uint32_t s = (uint32_t)cnt;
    const uint32_t km1 = (uint32_t)k - 1u;
    // groups: policy 2 puts the x = s mod (k-1) rightmost boundaries in a group of their own
    const uint32_t x = policy == 2 ? s % km1 : 0u;
    const uint32_t m = s == 0 ? 0u : (x ? 1u : 0u) + (s - x + km1 - 1u) / km1;
    if (threadIdx.x < s) sl[threadIdx.x] = list[threadIdx.x];
    __syncthreads();
    if (threadIdx.x < s) {
        const uint32_t b = sl[threadIdx.x];
        uint32_t rank = 0;  // boundaries to the left of b
        for (uint32_t j = 0; j < s; j++) rank += sl[j] < b ? 1u : 0u;
        const uint32_t t = s - 1u - rank;  // position from the right (0: the last boundary)
        const uint32_t g = x ? (t < x ? 0u : 1u + (t - x) / km1) : t / km1;  // group from the right
        powers[b] = (uint8_t)(0x80u | (m - g));
    }
    if (threadIdx.x == 0) {
        const unsigned long long bits = ctr[kCtrLevelBits];
        const uint32_t pmax = bits ? 63u - (uint32_t)__clzll((long long)bits) : 0u;
        // the depth and merge-cost scans hold powers 1..32 in 32-bit sets
        if (pmax + m > 32u) dev_fail(status, kDevTail);
        ctr[kCtrTailShift] = m;
        ctr[kCtrLevelBits] = 0;
    }
}

// Every boundary 1..r-1: a stack boundary keeps its label, any other power
// rises by m; rebuilds the bit set of powers that occur.
__global__ void __launch_bounds__(kTailThreads) k_tail_apply(uint8_t* __restrict__ powers, uint64_t* __restrict__ ctr) {
    __shared__ unsigned long long tmp[kTailThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t shift = (uint32_t)ctr[kCtrTailShift];
    const uint32_t groups = (uint32_t)ceil_div((uint64_t)r + 1, kTailItems);
    const uint32_t iters = (uint32_t)ceil_div(groups, (uint64_t)gridDim.x * blockDim.x);
    unsigned long long bits = 0;
    for (uint32_t it = 0; it < iters; it++) {
        const uint32_t gi = (it * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
        const uint32_t b0 = gi * kTailItems;
        if (gi >= groups || b0 > r) continue;
        uint4 w = load_word(powers, b0);
#pragma unroll
        for (int q = 0; q < kTailItems; q++) {
            const uint32_t b = b0 + q;
            if (b < 1 || b >= r) continue;
            const uint32_t p = byte_of(w, q);
            const uint32_t np = (p & 0x80u) ? (p & 0x7Fu) : p + shift;
            set_byte(w, q, np);
            bits |= 1ull << (np & 63u);
        }
        *reinterpret_cast<uint4*>(powers + b0) = w;
    }
    bits = block_reduce<kTailThreads>(bits, OpOrU64(), 0ull, tmp);
    if (threadIdx.x == 0 && bits) atomicOr(reinterpret_cast<unsigned long long*>(ctr + kCtrLevelBits), bits);
}

}  // namespace

void launch_tail(uint32_t r_bound, int k, int policy, uint8_t* orig_powers, const WsView& ws, cudaStream_t st) {
    const uint32_t tiles = (uint32_t)ceil_div((uint64_t)r_bound + 1, kMaskTile);
    const uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, 152 * 8);
    k_tail_tilemin<<<grid, kTailThreads, 0, st>>>(ws.powers, ws.counters, ws.mt_f);
    k_tail_tilescan<<<1, 1024, 0, st>>>(ws.counters, ws.mt_f, ws.mt_g);
    k_tail_mark<<<grid, kTailThreads, 0, st>>>(ws.powers, ws.counters, ws.mt_g, ws.tail_list, orig_powers);
    k_tail_assign<<<1, kTailCap, 0, st>>>(ws.powers, ws.counters, ws.tail_list, k, policy);
    const uint32_t groups = (uint32_t)ceil_div((uint64_t)r_bound + 1, kTailItems);
    const uint32_t agrid = (uint32_t)std::min<uint64_t>(ceil_div(groups, kTailThreads), 152 * 8);
    k_tail_apply<<<agrid, kTailThreads, 0, st>>>(ws.powers, ws.counters);
    g_launches += 5;
}

}  // namespace mps
