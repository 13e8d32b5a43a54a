// tree.cu -- the merge tree of Alg. 1 built from the boundary powers.
//
// Alg. 1 (KwayTree_k) splits a range of runs at every boundary of minimum
// power and recurses.  Unrolled, a node is a maximal group of equal-power
// boundaries not separated by any boundary of smaller power; it covers the
// runs between its delimiters L and R, the nearest boundaries of smaller
// power on either side (the virtual boundaries 0 and r have power 0).  Its
// parent owns whichever delimiter has the larger power (Alg. 1 recursed into
// that side last).  The nodes of power p are disjoint and depend only on
// nodes of larger power, so the tree executes level by level, p = max .. 1.
//
// Nearest-smaller queries run on a fan-out-32 min-tree over the u8 powers.
//
// Depths come from two scans.  The ancestors of a node are one node per
// distinct power among the "staircase" boundaries around it: the suffix
// minima of the powers to its left and the prefix minima to its right.  A
// segment is summarised by (bit set of its suffix-minimum values, its minimum);
// the summaries compose associatively:
//   F(XY) = (F_Y.bits | (F_X.bits & below(min_Y)), min(min_X, min_Y))
// and symmetrically for prefix minima.  Then
//   depth(node of B_j) = |(F(P_1..P_{j-1}) | G(P_{j+1}..P_{r-1})) & below(P_j)|,
//   depth(run i)       = |F(P_1..P_i) | G(P_{i+1}..P_{r-1})|,
// and B_j starts its node iff P_j is not among the suffix minima to its left.
// (Sec. 2.2: M = sum_i d_i L_i; Fact 3.2: depth(m(B_j)) <= P_j - 1.)
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

// ------------------------------------------------------------- min-tree

// Two levels of the min-tree at once: dst1[e] = min(src[32e .. 32e+31]) and
// dst2[e] = min(src[1024e .. 1024e+1023]), each written up to its padded
// length (a multiple of 32, 255 past the data).  Source level t holds
// ceil((r + 1) / 32^t) entries, r read on the device.  A thread reads 16
// source bytes; a block covers 4096 (128 dst1 and 4 dst2 entries) per step of
// a grid-stride loop.
__global__ void __launch_bounds__(256) k_mintree(const uint64_t* __restrict__ ctr, int t, const uint8_t* __restrict__ src,
                                                 uint8_t* __restrict__ dst1, uint8_t* __restrict__ dst2) {
    __shared__ uint32_t wmin[8];
    uint64_t len = (uint64_t)(uint32_t)ctr[kCtrR] + 1;
    for (int q = 0; q < t; q++) len = (len + 31) / 32;
    const uint32_t src_len = (uint32_t)len;
    const uint32_t dst1_len = (uint32_t)(((len + 31) / 32 + 31) / 32 * 32);
    const uint32_t dst2_len = (uint32_t)(((len + 1023) / 1024 + 31) / 32 * 32);
    const uint32_t nblk = (src_len + 4095) / 4096;
    for (uint32_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const uint32_t i0 = (blk * 256u + threadIdx.x) * 16u;
        uint32_t m = 255u;
        if (i0 < src_len) {
            const uint4 w = *reinterpret_cast<const uint4*>(src + i0);
            uint32_t x = __vminu4(__vminu4(w.x, w.y), __vminu4(w.z, w.w));
            if (i0 + 16u > src_len) {  // bytes past the data count as 255
                const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
                x = 0xFFFFFFFFu;
                for (uint32_t q = 0; q < 16u && i0 + q < src_len; q++) {
                    const uint32_t b = (wd[q >> 2] >> (8 * (q & 3))) & 0xFFu;
                    x = __vminu4(x, b * 0x01010101u);
                }
            }
            x = __vminu4(x, x >> 16);
            x = __vminu4(x, x >> 8);
            m = x & 0xFFu;
        }
        const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        const uint32_t m1 = min(m, __shfl_xor_sync(0xffffffffu, m, 1));  // 32 source bytes
        const uint32_t e1 = (blk * 256u + threadIdx.x) >> 1;
        if (!(lane & 1u) && e1 < dst1_len) dst1[e1] = (uint8_t)m1;
        if (dst2 != nullptr) {
            const uint32_t wm = __reduce_min_sync(0xffffffffu, m1);  // 512 source bytes
            if (lane == 0) wmin[warp] = wm;
            __syncthreads();
            if (threadIdx.x < 4) {
                const uint32_t e2 = blk * 4u + threadIdx.x;
                if (e2 < dst2_len) dst2[e2] = (uint8_t)min(wmin[2 * threadIdx.x], wmin[2 * threadIdx.x + 1]);
            }
            __syncthreads();
        }
    }
    if (dst2 != nullptr && blockIdx.x == 0)
        for (uint32_t q = nblk * 4u + threadIdx.x; q < dst2_len; q += 256u) dst2[q] = 255;
}

struct MinTree {
    const uint8_t* lv[kMinTreeLevels];
    int nl;
};

// Bit b set iff blk[b] < v (strict) or blk[b] <= v; blk is 32-byte aligned.
__device__ __forceinline__ uint32_t match32(const uint8_t* blk, uint32_t v, bool strict) {
    const uint4* p = reinterpret_cast<const uint4*>(blk);
    uint4 a = p[0], b = p[1];
    uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t vv = v * 0x01010101u;
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        uint32_t c = strict ? __vcmpltu4(w[q], vv) : __vcmpleu4(w[q], vv);
        uint32_t nib = ((c >> 7) & 1u) | ((c >> 14) & 2u) | ((c >> 21) & 4u) | ((c >> 28) & 8u);
        m |= nib << (4 * q);
    }
    return m;
}

// Nearest index l < i with P_l < v (strict) or P_l <= v.
__device__ uint32_t nsv_left(const MinTree& T, uint32_t i, uint32_t v, bool strict) {
    uint32_t pos = i;
    for (int t = 0; t < T.nl; t++) {
        uint32_t bs = pos & ~31u;
        uint32_t off = pos - bs;
        uint32_t m = off ? (match32(T.lv[t] + bs, v, strict) & (0xFFFFFFFFu >> (32 - off))) : 0u;
        if (m) {
            uint32_t j = bs + 31 - __clz(m);
            while (t > 0) {
                t--;
                uint32_t cm = match32(T.lv[t] + j * 32u, v, strict);
                j = j * 32u + 31 - __clz(cm);
            }
            return j;
        }
        pos = bs >> 5;
    }
    return kNone;
}

// Nearest index l > i with P_l < v (strict) or P_l <= v.
__device__ uint32_t nsv_right(const MinTree& T, uint32_t i, uint32_t v, bool strict) {
    uint32_t pos = i;
    for (int t = 0; t < T.nl; t++) {
        uint32_t bs = pos & ~31u;
        uint32_t off = pos - bs;
        uint32_t m = off < 31 ? (match32(T.lv[t] + bs, v, strict) & (0xFFFFFFFFu << (off + 1))) : 0u;
        if (m) {
            uint32_t j = bs + __ffs(m) - 1;
            while (t > 0) {
                t--;
                uint32_t cm = match32(T.lv[t] + j * 32u, v, strict);
                j = j * 32u + __ffs(cm) - 1;
            }
            return j;
        }
        pos = bs >> 5;
    }
    return kNone;
}

MinTree make_mintree(const WsView& ws) {
    MinTree T;
    for (int t = 0; t < kMinTreeLevels; t++) T.lv[t] = ws.lv[t];
    T.nl = ws.nlv;
    return T;
}

// ------------------------------------------------------------- masks

// A summary is (minimum power) << 32 | bit set of powers, bit p - 1 standing
// for power p (powers are 1..32 for n < 2^31; power 0, an array start, has no
// bit).  The identity has minimum 255 and no bits.
constexpr uint64_t kMaskIdentity = 255ull << 32;

// bits of the powers 1 .. m-1
__device__ __forceinline__ uint32_t below(uint32_t m) { return m <= 1 ? 0u : (m >= 33 ? ~0u : (~0u >> (33 - m))); }
__device__ __forceinline__ uint32_t mmin(uint64_t x) { return (uint32_t)(x >> 32); }
__device__ __forceinline__ uint32_t mbits(uint64_t x) { return (uint32_t)x; }
__device__ __forceinline__ uint64_t melem(uint32_t p) { return ((uint64_t)p << 32) | (p ? (1u << (p - 1)) : 0u); }

// suffix-minima summary, X then Y
struct OpF {
    __device__ unsigned long long operator()(unsigned long long X, unsigned long long Y) const {
        const uint32_t mx = mmin(X), my = mmin(Y);
        const uint32_t bits = mbits(Y) | (mbits(X) & below(my));
        return ((uint64_t)(mx < my ? mx : my) << 32) | bits;
    }
};
// prefix-minima summary, X then Y
struct OpG {
    __device__ unsigned long long operator()(unsigned long long X, unsigned long long Y) const {
        const uint32_t mx = mmin(X), my = mmin(Y);
        const uint32_t bits = mbits(X) | (mbits(Y) & below(mx));
        return ((uint64_t)(mx < my ? mx : my) << 32) | bits;
    }
};
// the same prefix-minima summary for a reverse-order scan: a follows b in scan order
struct OpGRev {
    __device__ unsigned long long operator()(unsigned long long A, unsigned long long B) const { return OpG()(B, A); }
};

constexpr int kMaskThreads = 256;
constexpr int kMaskItems = kMaskTile / kMaskThreads;

__global__ void __launch_bounds__(kMaskThreads) k_mask_reduce(const uint8_t* __restrict__ powers, const uint64_t* __restrict__ ctr,
                                                              unsigned long long* __restrict__ tf, unsigned long long* __restrict__ tg) {
    __shared__ unsigned long long tmp[kMaskThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t nb = r - 1;
    const uint32_t tiles = (uint32_t)ceil_div(max(nb, 1u), kMaskTile);
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t b0 = tile * kMaskTile + threadIdx.x * kMaskItems;
    unsigned long long f = kMaskIdentity, g = kMaskIdentity;
    if (b0 < nb) {
        // powers[b0 .. b0+31] (padded past r); boundary b is j = b + 1
        const uint4* p4 = reinterpret_cast<const uint4*>(powers + b0);
        const uint4 a = p4[0], c = p4[1];
        const uint32_t pw[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < kMaskItems; q++) {
            if (b0 + q < nb) {
                const uint64_t e = melem((pw[(q + 1) >> 2] >> (8 * ((q + 1) & 3))) & 0xFFu);
                f = OpF()(f, e);
                g = OpG()(g, e);
            }
        }
    }
    unsigned long long tot;
    block_scan_excl<kMaskThreads, false>(f, OpF(), kMaskIdentity, tmp, &tot);
    if (threadIdx.x == 0) tf[tile] = tot;
    block_scan_excl<kMaskThreads, false>(g, OpG(), kMaskIdentity, tmp, &tot);
    if (threadIdx.x == 0) tg[tile] = tot;
    }
}

__global__ void __launch_bounds__(1024) k_mask_scan(const unsigned long long* __restrict__ tf, const unsigned long long* __restrict__ tg,
                                                    const uint64_t* __restrict__ ctr, unsigned long long* __restrict__ fpre,
                                                    unsigned long long* __restrict__ gsuf) {
    __shared__ unsigned long long tmp[1024 / 32 + 1];
    const uint32_t nb = (uint32_t)ctr[kCtrR] - 1;
    const uint32_t tiles = (uint32_t)ceil_div(max(nb, 1u), kMaskTile);
    uint32_t per = (tiles + 1023) / 1024;
    uint32_t b = threadIdx.x * per, e = min(tiles, b + per);
    unsigned long long f = kMaskIdentity, g = kMaskIdentity;
    for (uint32_t t = b; t < e; t++) f = OpF()(f, tf[t]);
    for (uint32_t t = e; t > b; t--) g = OpG()(tg[t - 1], g);
    unsigned long long pf = block_scan_excl<1024, false>(f, OpF(), kMaskIdentity, tmp, nullptr);
    unsigned long long sg = block_scan_excl<1024, true>(g, OpGRev(), kMaskIdentity, tmp, nullptr);
    for (uint32_t t = b; t < e; t++) {
        fpre[t] = pf;
        pf = OpF()(pf, tf[t]);
    }
    for (uint32_t t = e; t > b; t--) {
        gsuf[t - 1] = sg;
        sg = OpG()(tg[t - 1], sg);
    }
}

// Smallest power v >= 1 whose inner nodes are provably at most T_max elements
// (255 if none).  Every interior boundary of a node of power v has power >= v,
// i.e. P2 > (v-1) log2 k (Def. 3.1 with P_k = ceil(P2 / log2 k)), so adjacent
// runs of the node have midpoints a/n that agree in their first (v-1) log2 k
// bits: all run midpoints of the node lie in one interval of n / k^(v-1)
// elements, and the node is smaller than that plus half of each end run, i.e.
// than n / k^(v-1) + (longest run).  (A batch takes its longest array for n.)
__device__ __forceinline__ uint32_t small_power(uint64_t nmax, uint64_t longest, uint32_t log2k, uint32_t tmax) {
    for (uint32_t v = 1; v < 64; v++) {
        const uint32_t sh = (v - 1) * log2k;
        const uint64_t span = sh >= 63 ? 1ull : ((nmax + (1ull << sh) - 1) >> sh);
        if (span + longest <= tmax) return v;
    }
    return 255u;
}

// Per boundary j = b + 1, node_info[b] = depth | query << 6 | start << 7, where
// start marks the first boundary of a node and query marks the starts the
// node pass must examine: roots (depth 0) and nodes of power below
// small_power().  Optionally writes the leaf depths, and adds to the counters
// the merge cost M = sum_i depth(run i) L_i (Sec. 2.2) and the number of nodes.
// Each thread holds 16 boundaries: 16-byte loads of powers and run starts and
// one 16-byte store of node_info.  With kArr (a batch whose caller asked for
// per-array costs) each run's term depth * L is also added to the cost of the
// array that holds it, arr_cost[a] for off[a] <= run start < off[a+1]: the
// tree of a batch has every array as a root, so a run's depth counts the
// merges inside its own array only and M of the array is Sec. 2.2's M of that
// array sorted alone.
template <bool kArr>
__global__ void __launch_bounds__(kMaskThreads, 4) k_mask_apply(const uint8_t* __restrict__ powers, uint64_t* __restrict__ ctr,
                                                             const uint32_t* __restrict__ rs,
                                                             const unsigned long long* __restrict__ fpre,
                                                             const unsigned long long* __restrict__ gsuf,
                                                             uint8_t* __restrict__ node_info, uint8_t* __restrict__ leaf_depth,
                                                             uint64_t n_single, uint32_t log2k, uint32_t tmax,
                                                             uint32_t* __restrict__ cand, uint32_t cand_cap,
                                                             const uint64_t* __restrict__ off, uint32_t m,
                                                             unsigned long long* __restrict__ arr_cost) {
    static_assert(kMaskItems == 16, "one 16-byte word of node_info per thread");
    __shared__ unsigned long long tmp[kMaskThreads / 32 + 1];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t nb = r - 1;
    const uint32_t tiles = (uint32_t)ceil_div(max(nb, 1u), kMaskTile);
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint32_t b0 = tile * kMaskTile + threadIdx.x * kMaskItems;
    const bool live = b0 < nb;
    // a final-collapse variant raised every power outside the final collapse by ctr[kCtrTailShift]
    const uint32_t vskip = small_power(n_single ? n_single : ctr[kCtrMaxLen], ctr[kCtrMaxRun], log2k, tmax) +
                           (uint32_t)ctr[kCtrTailShift];
    // powers[b0 .. b0+31] and rs[b0 .. b0+19] (both arrays are padded past r)
    uint32_t pw[8], rv[20];
    if (live) {
        const uint4* p4 = reinterpret_cast<const uint4*>(powers + b0);
        const uint4 a = p4[0], c = p4[1];
        pw[0] = a.x; pw[1] = a.y; pw[2] = a.z; pw[3] = a.w; pw[4] = c.x; pw[5] = c.y; pw[6] = c.z; pw[7] = c.w;
        const uint4* r4 = reinterpret_cast<const uint4*>(rs + b0);
#pragma unroll
        for (int q = 0; q < 5; q++) {
            const uint4 x = r4[q];
            rv[4 * q] = x.x; rv[4 * q + 1] = x.y; rv[4 * q + 2] = x.z; rv[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; q++) pw[q] = 0;
#pragma unroll
        for (int q = 0; q < 20; q++) rv[q] = 0;
    }
    // element of boundary b0 + q (the power of j = b0 + q + 1), identity past the end
    auto elem = [&](int q) -> unsigned long long {
        const uint32_t p = (pw[(q + 1) >> 2] >> (8 * ((q + 1) & 3))) & 0xFFu;
        return b0 + q < nb ? melem(p) : kMaskIdentity;
    };
    unsigned long long f = kMaskIdentity, g = kMaskIdentity;
#pragma unroll
    for (int q = 0; q < kMaskItems; q++) {
        const unsigned long long e = elem(q);
        f = OpF()(f, e);
        g = OpG()(g, e);
    }
    unsigned long long pf = block_scan_excl<kMaskThreads, false>(f, OpF(), kMaskIdentity, tmp, nullptr);
    unsigned long long sg = block_scan_excl<kMaskThreads, true>(g, OpGRev(), kMaskIdentity, tmp, nullptr);
    pf = OpF()(fpre[tile], pf);
    sg = OpG()(sg, gsuf[tile]);
    // bit sets of the right-side summaries per item (right to left)
    uint32_t rb[kMaskItems];
    uint32_t d0 = 0;  // depth of run 0 (thread holding boundary 1 only)
#pragma unroll
    for (int q = kMaskItems - 1; q >= 0; q--) {
        rb[q] = mbits(sg);
        const unsigned long long e = elem(q);
        if (q == 0 && b0 == 0) d0 = (uint32_t)__popc(mbits(OpG()(e, sg)));
        sg = OpG()(e, sg);
    }
    unsigned long long cost = 0, nodes = 0;
    // kArr: array a holds the run being counted, acost its running sum
    uint32_t a = 0;
    uint64_t a_end = 0;
    unsigned long long acost = 0;
    auto credit = [&](uint32_t start, unsigned long long t) {
        if (start >= a_end) {
            if (acost) atomicAdd(arr_cost + a, acost);
            acost = 0;
            do a_end = off[++a + 1]; while (start >= a_end);
        }
        acost += t;
    };
    if (kArr && live) {
        // last array a < m with off[a] <= first run start of this thread
        const uint32_t s0 = b0 == 0 ? rv[0] : rv[1];
        uint32_t lo = 0, hi = m - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= s0) lo = mid; else hi = mid - 1;
        }
        a = lo;
        a_end = off[a + 1];
    }
    uint32_t word[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < kMaskItems; q++) {
        const uint32_t b = b0 + q;
        const unsigned long long e = elem(q);
        if (b < nb) {
            const uint32_t j = b + 1;
            const uint32_t p = mmin(e);
            const uint32_t left = mbits(pf), right = rb[q];
            const uint32_t depth = __popc((left | right) & below(p));
            // power 0 marks an array start inside a batch: never a node boundary
            const uint32_t start = (p == 0 || ((left >> (p - 1)) & 1u)) ? 0u : 1u;
            const uint32_t query = start && (depth == 0 || p < vskip) ? 1u : 0u;
            word[q >> 2] |= (depth | (query << 6) | (start << 7)) << (8 * (q & 3));
            nodes += start;
            const uint32_t incl = mbits(OpF()(pf, e));
            const uint32_t dj = (uint32_t)__popc(incl | right);  // depth of run j
            if (j == 1) {
                const unsigned long long t0 = (unsigned long long)d0 * (rv[1] - rv[0]);
                cost += t0;
                if (kArr) credit(rv[0], t0);
                if (leaf_depth) leaf_depth[0] = (uint8_t)d0;
            }
            const unsigned long long tj = (unsigned long long)dj * (rv[q + 2] - rv[q + 1]);
            cost += tj;
            if (kArr) credit(rv[q + 1], tj);
            if (leaf_depth) leaf_depth[j] = (uint8_t)dj;
        }
        pf = OpF()(pf, e);
    }
    if (kArr && acost) atomicAdd(arr_cost + a, acost);
    if (live) *reinterpret_cast<uint4*>(node_info + b0) = make_uint4(word[0], word[1], word[2], word[3]);
    // append the marked starts to the candidate list of the node pass (one
    // atomic per warp that has any)
    {
        uint32_t qm = 0;  // bit q: boundary b0 + q is marked
#pragma unroll
        for (int q = 0; q < kMaskItems; q++) qm |= ((word[q >> 2] >> (8 * (q & 3) + 6)) & 1u) << q;
        const uint32_t cnt = __popc(qm);
        const uint32_t lane = threadIdx.x & 31u;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const uint32_t wtot = __shfl_sync(0xffffffffu, incl, 31);
        if (wtot) {
            uint32_t wbase = 0;
            if (lane == 31) wbase = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrCand), (unsigned long long)wtot);
            wbase = __shfl_sync(0xffffffffu, wbase, 31);
            uint32_t pos = wbase + incl - cnt;
            while (qm) {
                const uint32_t q = __ffs(qm) - 1;
                qm &= qm - 1;
                if (pos < cand_cap) cand[pos] = b0 + q + 1;
                pos++;
            }
        }
    }
    cost = block_reduce<kMaskThreads>(cost, OpAddU64(), 0ull, tmp);
    nodes = block_reduce<kMaskThreads>(nodes, OpAddU64(), 0ull, tmp);
    if (threadIdx.x == 0) {
        if (cost) atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrM), cost);
        if (nodes) atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrNodes), nodes);
    }
    }
}

// ------------------------------------------------------------- node pass

struct NodeShape {
    uint32_t L, R, d;
    uint32_t b[kMaxFanIn + 1];
};

__device__ __forceinline__ bool node_shape(const MinTree& T, const uint8_t* P, uint32_t j, uint32_t v, int k,
                                           NodeShape& s) {
    s.L = nsv_left(T, j, v, true);
    s.R = nsv_right(T, j, v, true);
    s.b[0] = s.L;
    s.b[1] = j;
    uint32_t cnt = 1, cur = j;
    bool ok = true;
    while (true) {
        uint32_t nx = nsv_right(T, cur, v, false);
        if (nx >= s.R) break;
        if ((int)cnt >= k - 1) { ok = false; break; }
        s.b[++cnt] = nx;
        cur = nx;
    }
    s.d = cnt + 1;
    s.b[s.d] = s.R;
    return ok;
}

// Finds the nodes larger than T_max among the node starts that k_mask_apply
// marked for a query and listed in `cand` (boundary indices j).  A large node becomes a level-merge record and appends each
// child that is an inner node of at most T_max elements to the list of fused
// subtrees (its parent is large, so it is maximal); a small root is a fused
// subtree too.
__global__ void __launch_bounds__(256) k_node_pass(MinTree T, int k, uint32_t tmax, uint32_t vmax,
                                                   const uint32_t* __restrict__ rs, const uint8_t* __restrict__ node_info,
                                                   uint64_t* __restrict__ ctr, LevelNode* __restrict__ nodes_raw, uint32_t nodes_cap,
                                                   uint4* __restrict__ fused_list, uint32_t fused_cap,
                                                   const uint32_t* __restrict__ cand, uint32_t cand_cap) {
    const uint8_t* P = T.lv[0];
    uint32_t* status = reinterpret_cast<uint32_t*>(ctr + kCtrStatus);
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint64_t ncand = ctr[kCtrCand];
    if (ncand > cand_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) dev_fail(status, kDevCapacity);
        return;
    }
    for (uint32_t ci = blockIdx.x * blockDim.x + threadIdx.x; ci < (uint32_t)ncand; ci += gridDim.x * blockDim.x) {
        {
            const uint32_t j = cand[ci];
            if (j == 0 || j >= r) {
                dev_fail(status, kDevRange);
                continue;
            }
            const uint32_t info = node_info[j - 1];
            const uint32_t v = P[j];
            const uint32_t depth = info & 0x3F;
            const uint32_t L = nsv_left(T, j, v, true);
            const uint32_t R = nsv_right(T, j, v, true);
            const uint32_t sL = rs[L], sR = rs[R];
            const uint32_t size = sR - sL;
            if (size > tmax) {
                // level merges are queued for powers 1..vmax only (a node of
                // power v is smaller than 3 n / k^(v-1)); anything else is a bug
                if (v > vmax + (uint32_t)ctr[kCtrTailShift]) dev_fail(status, kDevLevelBound);
                NodeShape s;
                if (!node_shape(T, P, j, v, k, s)) dev_fail(status, kDevDegree);
                uint32_t slot = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrHbmTotal), 1ull);
                if (slot < nodes_cap) {
                    LevelNode nd;
                    nd.sL = sL; nd.sR = sR; nd.unit_off = 0; nd.nunits = 0;
#pragma unroll
                    for (int c = 0; c <= kMaxFanIn; c++) nd.b[c] = c <= (int)s.d ? s.b[c] : 0u;
                    nd.power = (uint8_t)v; nd.depth = (uint8_t)depth; nd.degree = (uint8_t)s.d; nd.pad = 0;
                    nd.split_off = nd.nsplit = 0;
                    nodes_raw[slot] = nd;
                } else {
                    dev_fail(status, kDevCapacity);
                }
                atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrHbmCount + v), 1ull);
                atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrHbmSize + v), (unsigned long long)size);
                // Consecutive small inner children share one fused tile while
                // they fit: the tile carries the node's power v as a floor, so
                // its boundaries between the siblings (power v) stay delimiters
                // and only levels above v are merged.
                uint32_t ga = 0, ge = 0, gsz = 0;  // open group: runs [ga, ge), gsz elements
                for (uint32_t c = 0; c <= s.d; c++) {
                    bool take = false;
                    uint32_t a = 0, e = 0, cs = 0;
                    if (c < s.d) {
                        a = s.b[c];
                        e = s.b[c + 1];
                        cs = rs[e] - rs[a];
                        take = e - a >= 2 && cs <= tmax;
                    }
                    if (gsz && !(take && a == ge && gsz + cs <= tmax)) {
                        uint32_t fs = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrFrontier), 1ull);
                        if (fs < fused_cap) fused_list[fs] = make_uint4(ga, ge, depth + 1, v);
                        else dev_fail(status, kDevCapacity);
                        gsz = 0;
                    }
                    if (take) {
                        if (!gsz) ga = a;
                        ge = e;
                        gsz += cs;
                    }
                }
            } else if (P[L] == 0 && P[R] == 0) {
                // a root (of the array, or of one array of a batch) that fits a fused tile
                uint32_t fs = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrFrontier), 1ull);
                if (fs < fused_cap) fused_list[fs] = make_uint4(L, R, 0u, 0u);
                else dev_fail(status, kDevCapacity);
            }
        }
    }
}

// Copies level-merge nodes into per-power buckets (order within a bucket is
// irrelevant: nodes of one power are disjoint).
__global__ void k_bucket(const LevelNode* __restrict__ raw, const uint32_t* __restrict__ level_off,
                         uint64_t* __restrict__ ctr, LevelNode* __restrict__ out, uint32_t cap) {
    const uint32_t total = min((uint32_t)ctr[kCtrHbmTotal], cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        LevelNode nd = raw[i];
        uint32_t slot = (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(ctr + kCtrHbmFill + nd.power), 1ull);
        // the per-power counts include nodes the node pass could not store
        // (it reported that); nothing is written past the capacity
        const uint32_t at = level_off[nd.power] + slot;
        if (at < cap) out[at] = nd;
    }
}

// Exclusive offsets of the per-power node buckets (one thread).  Also caps
// the fused-subtree count at the list's capacity, so that the fused merge,
// which takes its work count from the device, never reads past the list (the
// node pass reported any overflow as a device status).
__global__ void k_level_offsets(uint64_t* __restrict__ ctr, uint32_t* __restrict__ off, uint32_t fused_cap) {
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int p = 0; p < kMaxLevels; p++) {
            off[p] = acc;
            acc += (uint32_t)ctr[kCtrHbmCount + p];
        }
        if (ctr[kCtrFrontier] > fused_cap) ctr[kCtrFrontier] = fused_cap;
    }
}

// ------------------------------------------------------------- tree dump

// node_first for every boundary; canonical rank is computed by k_dump_rank.
__global__ void __launch_bounds__(256) k_dump_node_first(MinTree T, const uint64_t* __restrict__ ctr,
                                                         const uint8_t* __restrict__ node_info,
                                                         uint32_t* __restrict__ node_first) {
    const uint8_t* P = T.lv[0];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) node_first[0] = 0;
    if (j == 0 || j >= r) return;
    if (node_info[j - 1] & 0x80) {
        node_first[j] = j;
    } else {
        uint32_t v = P[j];
        uint32_t L = nsv_left(T, j, v, true);
        node_first[j] = nsv_right(T, L, v, false);
    }
}

// Per-tile histograms of node-start powers (tile = kMaskTile boundaries).
__global__ void __launch_bounds__(256) k_dump_hist(const uint8_t* __restrict__ P, const uint8_t* __restrict__ node_info,
                                                   const uint64_t* __restrict__ ctr, uint32_t* __restrict__ hist) {
    const uint32_t r = (uint32_t)ctr[kCtrR];
    __shared__ uint32_t h[kMaxLevels];
    if (threadIdx.x < kMaxLevels) h[threadIdx.x] = 0;
    __syncthreads();
    uint32_t base = blockIdx.x * kMaskTile;
    for (uint32_t q = threadIdx.x; q < kMaskTile; q += blockDim.x) {
        uint32_t j = base + q + 1;
        if (j < r && (node_info[j - 1] & 0x80)) atomicAdd(&h[P[j]], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kMaxLevels) hist[(size_t)blockIdx.x * kMaxLevels + threadIdx.x] = h[threadIdx.x];
}

// Turns the histograms into exclusive offsets in (power, tile) order.  One block.
__global__ void __launch_bounds__(1024) k_dump_hist_scan(uint32_t* __restrict__ hist, uint32_t tiles) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t p = 0; p < (uint32_t)kMaxLevels; p++) {
        for (uint32_t t0 = 0; t0 < tiles; t0 += 1024) {
            uint32_t t = t0 + threadIdx.x;
            uint32_t v = t < tiles ? hist[(size_t)t * kMaxLevels + p] : 0u;
            uint32_t tot;
            uint32_t ex = block_sum_excl<1024>(v, tmp, &tot);
            uint32_t c = carry;
            if (t < tiles) hist[(size_t)t * kMaxLevels + p] = c + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry = c + tot;
            __syncthreads();
        }
    }
}

// Canonical rank of every node start: starts of power p in boundary order.
// Within a tile, a warp walks its boundaries in order with ballots.
__global__ void __launch_bounds__(256) k_dump_rank(const uint8_t* __restrict__ P, const uint8_t* __restrict__ node_info,
                                                   const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ hist,
                                                   uint32_t* __restrict__ canon_idx) {
    const uint32_t r = (uint32_t)ctr[kCtrR];
    __shared__ uint32_t run[kMaxLevels];
    if (threadIdx.x < kMaxLevels) run[threadIdx.x] = hist[(size_t)blockIdx.x * kMaxLevels + threadIdx.x];
    __syncthreads();
    // one warp walks the whole tile in order, 32 boundaries per step
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    uint32_t base = blockIdx.x * kMaskTile;
    for (uint32_t q0 = 0; q0 < (uint32_t)kMaskTile; q0 += 32) {
        uint32_t j = base + q0 + lane + 1;
        bool st = j < r && (node_info[j - 1] & 0x80);
        uint32_t p = st ? P[j] : 0xFFu;
        uint32_t peers = __match_any_sync(0xffffffffu, p);
        uint32_t below_me = __popc(peers & ((1u << lane) - 1));
        uint32_t cnt = __popc(peers);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t basep = 0;
        if (st) basep = run[p];
        __syncwarp();
        if (st) canon_idx[j] = basep + below_me;
        if (st && (uint32_t)lane == leader) run[p] = basep + cnt;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_dump_nodes(MinTree T, const uint64_t* __restrict__ ctr, int k, const uint32_t* __restrict__ rs,
                                                    const uint8_t* __restrict__ node_info, const uint32_t* __restrict__ canon_idx,
                                                    const uint32_t* __restrict__ node_first, uint32_t* __restrict__ out_nodes,
                                                    uint32_t* __restrict__ status) {
    const uint8_t* P = T.lv[0];
    const uint32_t r = (uint32_t)ctr[kCtrR];
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (j >= r || !(node_info[j - 1] & 0x80)) return;
    uint32_t v = P[j];
    NodeShape s;
    if (!node_shape(T, P, j, v, k, s)) dev_fail(status, kDevDegree);
    uint32_t parent = kNone;
    uint32_t pl = P[s.L], pr = P[s.R];
    if (pl != 0 || pr != 0) {
        uint32_t q = pl >= pr ? s.L : s.R;
        parent = canon_idx[node_first[q]];
    }
    uint32_t idx = canon_idx[j];
    uint32_t* o = out_nodes + (size_t)idx * 4;
    o[0] = s.L;
    o[1] = s.R;
    o[2] = v | (s.d << 8);
    o[3] = parent;
}

// Copies the run structure of a sort to the caller's tree arrays (r read on
// the device): run_starts[0..r], run_desc[0..r), powers[0..r], and, for an
// input of one run (no boundary, so no depth written by the depth scan),
// leaf_depth[0] = 0; block 0 writes counts = {r, nodes, distinct powers, M}.
__global__ void __launch_bounds__(256) k_tree_arrays(const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs,
                                                     const uint8_t* __restrict__ rdesc, const uint8_t* __restrict__ P,
                                                     uint32_t* __restrict__ o_rs, uint8_t* __restrict__ o_rd,
                                                     uint8_t* __restrict__ o_p, uint8_t* __restrict__ o_leaf,
                                                     uint64_t* __restrict__ o_counts) {
    const uint32_t r = (uint32_t)ctr[kCtrR];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= r; i += gridDim.x * blockDim.x) {
        if (o_rs) o_rs[i] = rs[i];
        if (o_rd && i < r) o_rd[i] = rdesc[i];
        if (o_p) o_p[i] = P[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (o_leaf && r == 1) o_leaf[0] = 0;
        if (o_counts) {
            o_counts[0] = r;
            o_counts[1] = ctr[kCtrNodes];
            o_counts[2] = (uint64_t)__popcll((long long)ctr[kCtrLevelBits]);
            o_counts[3] = ctr[kCtrM];
        }
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

void launch_mintree(uint32_t r_bound, const WsView& ws, cudaStream_t st) {
    // ws.nlv levels for up to r_bound runs; each kernel sizes its levels from r
    for (int t = 0; t + 1 < ws.nlv; t += 2) {
        const uint32_t src_bound = ws.lv_len[t];
        const uint32_t blocks = (uint32_t)std::min<uint64_t>((src_bound + 4095) / 4096, 152 * 8);
        uint8_t* dst2 = (t + 2 < ws.nlv) ? ws.lv[t + 2] : nullptr;
        k_mintree<<<blocks, 256, 0, st>>>(ws.counters, t, ws.lv[t], ws.lv[t + 1], dst2);
        g_launches += 1;
    }
}

void launch_masks(uint32_t r_bound, bool dump_leaf, uint8_t* leaf_depth, uint64_t n, int k, uint32_t tmax, const WsView& ws,
                  cudaStream_t st) {
    // tiles of kMaskTile boundaries for up to r_bound runs; the kernels loop over the tiles of the actual r
    const uint32_t nb = r_bound > 1 ? r_bound - 1 : 1;
    const uint32_t tiles = (uint32_t)ceil_div(nb, kMaskTile);
    const uint32_t grid = std::min<uint32_t>(tiles, 152 * 32);
    k_mask_reduce<<<grid, kMaskThreads, 0, st>>>(ws.powers, ws.counters, ws.mt_f, ws.mt_g);
    k_mask_scan<<<1, 1024, 0, st>>>(ws.mt_f, ws.mt_g, ws.counters, ws.mt_fpre, ws.mt_gsuf);
    const uint32_t log2k = (uint32_t)__builtin_ctz((unsigned)k);
    if (ws.batch_cost)
        k_mask_apply<true><<<grid, kMaskThreads, 0, st>>>(
            ws.powers, ws.counters, ws.run_starts, ws.mt_fpre, ws.mt_gsuf, ws.node_info, dump_leaf ? leaf_depth : nullptr,
            0ull, log2k, tmax, ws.canon_idx, ws.cand_cap, ws.batch_off, ws.batch_m,
            reinterpret_cast<unsigned long long*>(ws.batch_cost));
    else
        k_mask_apply<false><<<grid, kMaskThreads, 0, st>>>(
            ws.powers, ws.counters, ws.run_starts, ws.mt_fpre, ws.mt_gsuf, ws.node_info, dump_leaf ? leaf_depth : nullptr,
            ws.batch_off ? 0ull : n, log2k, tmax, ws.canon_idx, ws.cand_cap, nullptr, 0u, nullptr);
    g_launches += 3;
}

void launch_node_pass(uint32_t r, int k, uint32_t tmax, uint32_t vmax, const WsView& ws, cudaStream_t st) {
    (void)r;
    k_node_pass<<<152 * 4, 256, 0, st>>>(make_mintree(ws), k, tmax, vmax, ws.run_starts, ws.node_info, ws.counters, ws.nodes_raw,
                                         ws.nodes_cap, ws.fused_list, ws.fused_cap, ws.canon_idx, ws.cand_cap);
    g_launches += 1;
}

void launch_bucket(uint32_t total_bound, const WsView& ws, cudaStream_t st) {
    k_level_offsets<<<1, 32, 0, st>>>(ws.counters, ws.level_off, ws.fused_cap);
    uint32_t blocks = (uint32_t)std::min<uint64_t>(ceil_div(std::max<uint32_t>(total_bound, 1), 256), 152 * 8);
    k_bucket<<<blocks, 256, 0, st>>>(ws.nodes_raw, ws.level_off, ws.counters, ws.nodes_lvl, ws.nodes_cap);
    g_launches += 2;
}

void launch_tree_dump(uint32_t r_bound, int k, const WsView& ws, uint32_t* node_first, void* nodes, cudaStream_t st) {
    const uint32_t nb = r_bound > 0 ? r_bound - 1 : 0;
    const uint32_t tiles = (uint32_t)std::max<uint64_t>(1, ceil_div(nb, kMaskTile));
    MinTree T = make_mintree(ws);
    k_dump_node_first<<<(uint32_t)ceil_div(std::max<uint32_t>(r_bound, 1), 256), 256, 0, st>>>(T, ws.counters, ws.node_info,
                                                                                                 node_first);
    k_dump_hist<<<tiles, 256, 0, st>>>(ws.powers, ws.node_info, ws.counters, ws.hist);
    k_dump_hist_scan<<<1, 1024, 0, st>>>(ws.hist, tiles);
    k_dump_rank<<<tiles, 256, 0, st>>>(ws.powers, ws.node_info, ws.counters, ws.hist, ws.canon_idx);
    if (nodes)
        k_dump_nodes<<<(uint32_t)std::max<uint64_t>(1, ceil_div(nb, 256)), 256, 0, st>>>(
            T, ws.counters, k, ws.run_starts, ws.node_info, ws.canon_idx, node_first, reinterpret_cast<uint32_t*>(nodes),
            reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus));
    g_launches += nodes ? 5 : 4;
}

void launch_tree_arrays(uint32_t r_bound, const WsView& ws, const uint8_t* desc_src, uint32_t* run_starts,
                        uint8_t* run_desc, uint8_t* powers, uint8_t* leaf_depth, uint64_t* counts, cudaStream_t st) {
    const uint32_t blocks = (uint32_t)std::min<uint64_t>(ceil_div((uint64_t)r_bound + 1, 256), 152 * 8);
    k_tree_arrays<<<blocks, 256, 0, st>>>(ws.counters, ws.run_starts, desc_src, ws.powers, run_starts, run_desc, powers,
                                          leaf_depth, counts);
    g_launches += 1;
}

}  // namespace mps
