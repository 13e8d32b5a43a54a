// merge.cu -- execution of the merge tree (Sec. 2.2) as stable k-way merges.
//
// A node of degree d merges its d children (left to right) into one sorted
// run; equal keys come out from the leftmost child first, as in the paper's
// tournament whose matches prefer the left entrant ("<=", Sec. 4 "Tournament
// tree").  On chip, a d-way merge is played exactly as that tournament is
// shaped: a balanced binary bracket, children (0,1), (2,3), ... meet in round
// 0, the winners' runs meet in round 1, and so on.  Each round is a set of
// stable 2-way merges in shared memory, one merge-path search per thread.
// Global memory sees each element once per node: one read of the children
// and one write of the node's output, which is the merge cost M of Sec. 2.2
// counted in elements moved.
//
// Two kernels execute the tree:
//   * k_fused: every maximal subtree of at most T_max elements (a "frontier"
//     node with its descendants) is loaded once into shared memory, all of
//     its levels are merged there, and its output is written once;
//   * k_level_*: the nodes above the frontier, one launch per power level
//     (p = max .. 1).  Each node is cut into work units at splitters: every
//     T_s-th element of every child.  A splitter's position in each other
//     child is a binary search under the total order (key, child, position),
//     which makes every unit a contiguous slice of every child and of the
//     output (the co-ranking of merge-path merging, taken to d children).
// Node outputs alternate between the output array (even depth) and the
// temporary array (odd depth), so the root lands in the output; leaves are
// read from the input, strictly descending runs reversed on the fly.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

constexpr int kMergeThreads = 512;
constexpr int kIPT = 8;
constexpr uint32_t kNoMid = 0xFFFFu;
// boundary-list entries one thread holds while compacting: ceil((C/2 + 8) / 512)
constexpr int kKeepMax = 24;

// One pass of stable 2-way merges over [0, len): segment i covers
// [seg_start[i], seg_start[i+1]) and merges its halves at seg_mid[i], or is
// copied when seg_mid[i] == kNoMid.
template <typename K, bool V>
__device__ __forceinline__ void merge_pass(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
                                           uint32_t* __restrict__ vdst, uint32_t len, const uint16_t* __restrict__ seg_start,
                                           const uint16_t* __restrict__ seg_mid, uint32_t ns) {
    for (uint32_t base = threadIdx.x * kIPT; base < len; base += kMergeThreads * kIPT) {
        uint32_t o = base;
        const uint32_t oe = min(base + (uint32_t)kIPT, len);
        uint32_t lo = 0, hi = ns;
        while (hi - lo > 1) {
            uint32_t m = (lo + hi) >> 1;
            if (seg_start[m] <= o) lo = m; else hi = m;
        }
        uint32_t i = lo;
        while (o < oe) {
            const uint32_t s = seg_start[i], e = seg_start[i + 1], m = seg_mid[i];
            const uint32_t stop = min(e, oe);
            if (m == kNoMid) {
                for (; o < stop; o++) {
                    dst[o] = src[o];
                    if (V) vdst[o] = vsrc[o];
                }
            } else {
                const uint32_t na = m - s, nbn = e - m, diag = o - s;
                uint32_t l = diag > nbn ? diag - nbn : 0u, h = min(diag, na);
                while (l < h) {
                    uint32_t mid = (l + h) >> 1;
                    if (src[s + mid] <= src[m + diag - 1 - mid]) l = mid + 1; else h = mid;
                }
                uint32_t ia = s + l, ib = m + diag - l;
                K ka = ia < m ? src[ia] : K(0);
                K kb = ib < e ? src[ib] : K(0);
                for (; o < stop; o++) {
                    bool take_a = ia < m && (ib >= e || ka <= kb);
                    if (take_a) {
                        dst[o] = ka;
                        if (V) vdst[o] = vsrc[ia];
                        ia++;
                        ka = ia < m ? src[ia] : K(0);
                    } else {
                        dst[o] = kb;
                        if (V) vdst[o] = vsrc[ib];
                        ib++;
                        kb = ib < e ? src[ib] : K(0);
                    }
                }
            }
            i++;
        }
    }
}

// Entry of the shared-memory boundary list: bits 0..15 element offset,
// 16..23 power (0 = never merged here), 24..31 index q within its group.
__device__ __forceinline__ uint32_t be_off(uint32_t e) { return e & 0xFFFFu; }
__device__ __forceinline__ uint32_t be_pow(uint32_t e) { return (e >> 16) & 0xFFu; }
__device__ __forceinline__ uint32_t be_q(uint32_t e) { return e >> 24; }

// Segmented count: bit 31 = group reset, low bits = equal-power boundaries seen.
struct OpSegCount {
    __device__ uint32_t operator()(uint32_t X, uint32_t Y) const {
        return (Y & 0x80000000u) ? Y : ((X & 0x80000000u) | ((X & 0x7FFFFFFFu) + Y));
    }
};

template <typename K, bool V>
struct SmemLayout {
    static __host__ __device__ size_t bytes(uint32_t C) {
        uint32_t bmax = C / 2 + 8;
        return (size_t)2 * C * sizeof(K) + (V ? (size_t)2 * C * 4 : 0) + (size_t)2 * bmax * 4;
    }
};

template <typename K, bool V>
__global__ void __launch_bounds__(kMergeThreads, 1)
    k_fused(const K* __restrict__ leaf, const uint32_t* __restrict__ vleaf, K* __restrict__ out0, K* __restrict__ out1,
            uint32_t* __restrict__ vout0, uint32_t* __restrict__ vout1, const uint32_t* __restrict__ rs,
            const uint8_t* __restrict__ rdesc, const uint8_t* __restrict__ P, const uint32_t* __restrict__ fr_end,
            const uint8_t* __restrict__ fr_depth, const uint32_t* __restrict__ first_run, uint32_t C, int k,
            uint32_t* __restrict__ status) {
    extern __shared__ uint4 smem_raw[];
    const uint32_t BMAX = C / 2 + 8;
    K* kA = reinterpret_cast<K*>(smem_raw);
    K* kB = kA + C;
    uint32_t* vA = V ? reinterpret_cast<uint32_t*>(kB + C) : nullptr;
    uint32_t* vB = V ? vA + C : nullptr;
    uint32_t* bl0 = V ? (vB + C) : reinterpret_cast<uint32_t*>(kB + C);
    uint32_t* bl1 = bl0 + BMAX;
    __shared__ uint32_t fl_lo[kMaxFrontierPerWindow];
    __shared__ uint32_t fl_hi[kMaxFrontierPerWindow];
    __shared__ uint32_t stmp[kMergeThreads / 32 + 1];
    __shared__ uint32_t sh_total;

    const uint32_t tid = threadIdx.x;
    const uint32_t ra = first_run[blockIdx.x], rb = first_run[blockIdx.x + 1];
    if (ra >= rb) return;

    // ---- 1. frontier nodes starting in this window (ordered compaction)
    const uint32_t nw = rb - ra;
    uint32_t per = (nw + kMergeThreads - 1) / kMergeThreads;
    uint32_t w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
    uint32_t cnt = 0;
    for (uint32_t q = w0; q < w1; q++) cnt += fr_end[ra + q] != 0;
    uint32_t F;
    uint32_t pos = block_sum_excl<kMergeThreads>(cnt, stmp, &F);
    if (F == 0) return;
    if (F > (uint32_t)kMaxFrontierPerWindow) {
        if (tid == 0) dev_fail(status, kDevCapacity);
        return;
    }
    for (uint32_t q = w0; q < w1; q++) {
        uint32_t R = fr_end[ra + q];
        if (R) {
            fl_lo[pos] = ra + q;
            fl_hi[pos] = R | ((uint32_t)(fr_depth[ra + q] & 1u) << 31);
            pos++;
        }
    }
    __syncthreads();
    const uint32_t lo_run = fl_lo[0];
    const uint32_t hi_run = fl_hi[F - 1] & 0x7FFFFFFFu;
    const uint32_t s_lo = rs[lo_run];
    const uint32_t len = rs[hi_run] - s_lo;
    if (len > C) {
        if (tid == 0) dev_fail(status, kDevRange);
        return;
    }
    const uint32_t nruns = hi_run - lo_run;
    const uint32_t nb = nruns - 1;

    // ---- 2. boundary list; boundaries outside every frontier node never merge
    int8_t* mk = reinterpret_cast<int8_t*>(kB);
    for (uint32_t e = tid; e < nb; e += kMergeThreads) mk[e] = 0;
    __syncthreads();
    for (uint32_t f = tid; f < F; f += kMergeThreads) {
        uint32_t L = fl_lo[f], R = fl_hi[f] & 0x7FFFFFFFu;
        mk[L - lo_run] = 1;
        if (R - lo_run - 1 < nb) mk[R - lo_run - 1] = -1;
    }
    __syncthreads();
    per = (nb + kMergeThreads - 1) / kMergeThreads;
    uint32_t e0 = min(nb, tid * per), e1 = min(nb, e0 + per);
    {
        uint32_t s = 0;
        for (uint32_t e = e0; e < e1; e++) s += (uint32_t)(int32_t)mk[e];
        uint32_t run = block_sum_excl<kMergeThreads>(s, stmp, nullptr);
        for (uint32_t e = e0; e < e1; e++) {
            run += (uint32_t)(int32_t)mk[e];
            uint32_t j = lo_run + 1 + e;
            uint32_t p = (int32_t)run > 0 ? P[j] : 0u;
            bl0[e] = (rs[j] - s_lo) | (p << 16);
        }
    }
    // frontier ranges as element offsets (+ output parity)
    __syncthreads();
    for (uint32_t f = tid; f < F; f += kMergeThreads) {
        uint32_t L = fl_lo[f], h = fl_hi[f];
        fl_lo[f] = rs[L] - s_lo;
        fl_hi[f] = (rs[h & 0x7FFFFFFFu] - s_lo) | (h & 0x80000000u);
    }

    // ---- 3. load the keys, then reverse the strictly descending runs
    for (uint32_t x = tid; x < len; x += kMergeThreads) {
        kA[x] = leaf[s_lo + x];
        if (V) vA[x] = vleaf[s_lo + x];
    }
    uint8_t* dflag = reinterpret_cast<uint8_t*>(bl1);
    for (uint32_t q = tid; q < nruns; q += kMergeThreads) dflag[q] = rdesc[lo_run + q];
    __syncthreads();
    {
        uint32_t pe = (len + kMergeThreads - 1) / kMergeThreads;
        uint32_t x0 = min(len, tid * pe), x1 = min(len, x0 + pe);
        if (x0 < x1) {
            uint32_t lo = 0, hi = nb;  // runs before x0: boundaries with offset <= x0
            while (lo < hi) {
                uint32_t m = (lo + hi) >> 1;
                if (be_off(bl0[m]) <= x0) lo = m + 1; else hi = m;
            }
            uint32_t rho = lo;
            uint32_t rs0 = rho ? be_off(bl0[rho - 1]) : 0u;
            uint32_t re0 = rho < nb ? be_off(bl0[rho]) : len;
            for (uint32_t x = x0; x < x1; x++) {
                while (x >= re0) {
                    rho++;
                    rs0 = re0;
                    re0 = rho < nb ? be_off(bl0[rho]) : len;
                }
                uint32_t src = dflag[rho] ? (rs0 + re0 - 1 - x) : x;
                kB[x] = kA[src];
                if (V) vB[x] = vA[src];
            }
        }
    }
    __syncthreads();
    K* cur = kB;
    K* oth = kA;
    uint32_t* vcur = vB;
    uint32_t* voth = vA;

    // ---- 4. levels of the subtrees, largest power first
    uint32_t pmax = 0, pmin = 255;
    for (uint32_t e = e0; e < e1; e++) {
        uint32_t p = be_pow(bl0[e]);
        if (p) { pmax = max(pmax, p); pmin = min(pmin, p); }
    }
    pmax = block_reduce<kMergeThreads>(pmax, OpMax32(), 0u, stmp);
    pmin = 255u - block_reduce<kMergeThreads>(255u - pmin, OpMax32(), 0u, stmp);
    uint32_t na = nb;
    uint16_t* seg_start = reinterpret_cast<uint16_t*>(bl1);
    uint16_t* seg_mid = seg_start + BMAX + 2;

    for (uint32_t p = pmax; p >= pmin && p >= 1; p--) {
        per = (na + kMergeThreads - 1) / kMergeThreads;
        e0 = min(na, tid * per);
        e1 = min(na, e0 + per);
        // group index q of every power-p boundary
        uint32_t acc = 0;
        for (uint32_t e = e0; e < e1; e++) {
            uint32_t pw = be_pow(bl0[e]);
            uint32_t x = pw < p ? 0x80000000u : (pw == p ? 1u : 0u);
            acc = OpSegCount()(acc, x);
        }
        uint32_t pre = block_scan_excl<kMergeThreads, false>(acc, OpSegCount(), 0u, stmp, nullptr);
        uint32_t neq = 0;
        for (uint32_t e = e0; e < e1; e++) {
            uint32_t v = bl0[e];
            uint32_t pw = be_pow(v);
            uint32_t x = pw < p ? 0x80000000u : (pw == p ? 1u : 0u);
            pre = OpSegCount()(pre, x);
            if (pw == p) {
                bl0[e] = (v & 0x00FFFFFFu) | ((pre & 0x7FFFFFFFu) << 24);
                neq++;
            }
        }
        neq = block_reduce<kMergeThreads>(neq, OpAdd32(), 0u, stmp);
        if (neq == 0) continue;
        // tournament rounds
        for (uint32_t t = 0; (1u << t) < (uint32_t)k; t++) {
            uint32_t nd = 0, nm = 0;
            for (uint32_t e = e0; e < e1; e++) {
                uint32_t v = bl0[e];
                uint32_t pw = be_pow(v);
                uint32_t cz = pw == p ? (uint32_t)__ffs(be_q(v)) - 1 : 0u;
                nd += (pw < p) || (pw == p && cz > t);
                nm += (pw == p && cz == t);
            }
            uint32_t ndel;
            uint32_t dpos = block_sum_excl<kMergeThreads>(nd, stmp, &ndel);
            uint32_t nmt = block_reduce<kMergeThreads>(nm, OpAdd32(), 0u, stmp);
            if (nmt == 0) break;
            const uint32_t ns = ndel + 1;
            for (uint32_t i = tid; i < ns; i += kMergeThreads) seg_mid[i] = (uint16_t)kNoMid;
            if (tid == 0) {
                seg_start[0] = 0;
                seg_start[ns] = (uint16_t)len;
            }
            for (uint32_t e = e0; e < e1; e++) {
                uint32_t v = bl0[e];
                uint32_t pw = be_pow(v);
                uint32_t cz = pw == p ? (uint32_t)__ffs(be_q(v)) - 1 : 0u;
                if ((pw < p) || (pw == p && cz > t)) seg_start[1 + dpos++] = (uint16_t)be_off(v);
            }
            __syncthreads();
            dpos -= nd;
            for (uint32_t e = e0; e < e1; e++) {
                uint32_t v = bl0[e];
                uint32_t pw = be_pow(v);
                uint32_t cz = pw == p ? (uint32_t)__ffs(be_q(v)) - 1 : 0u;
                bool del = (pw < p) || (pw == p && cz > t);
                if (pw == p && cz == t) seg_mid[dpos] = (uint16_t)be_off(v);
                dpos += del;
            }
            __syncthreads();
            merge_pass<K, V>(cur, oth, vcur, voth, len, seg_start, seg_mid, ns);
            __syncthreads();
            K* tk = cur; cur = oth; oth = tk;
            uint32_t* tv = vcur; vcur = voth; voth = tv;
        }
        // drop the boundaries consumed at this level
        uint32_t keep[kKeepMax];
        uint32_t nk = 0;
        for (uint32_t e = e0; e < e1; e++) {
            uint32_t v = bl0[e];
            if (be_pow(v) < p) keep[nk++] = v & 0x00FFFFFFu;
        }
        uint32_t ntot;
        uint32_t kpos = block_sum_excl<kMergeThreads>(nk, stmp, &ntot);
        for (uint32_t q = 0; q < nk; q++) bl0[kpos + q] = keep[q];
        na = ntot;
        __syncthreads();
    }

    // ---- 5. write every frontier node's output
    for (uint32_t x = tid; x < len; x += kMergeThreads) {
        uint32_t lo = 0, hi = F;
        while (hi - lo > 1) {
            uint32_t m = (lo + hi) >> 1;
            if (fl_lo[m] <= x) lo = m; else hi = m;
        }
        uint32_t h = fl_hi[lo];
        if (x >= fl_lo[lo] && x < (h & 0x7FFFFFFFu)) {
            K* o = (h >> 31) ? out1 : out0;
            o[s_lo + x] = cur[x];
            if (V) {
                uint32_t* vo = (h >> 31) ? vout1 : vout0;
                vo[s_lo + x] = vcur[x];
            }
        }
    }
}

// ------------------------------------------------------------ level merges

struct Child {
    uint32_t base;   // first element of the child in its buffer
    uint32_t len;
    uint32_t leaf;   // read from the input (1) or from a node buffer (0)
    uint32_t rev;    // leaf was strictly descending: read backwards
};

__device__ __forceinline__ Child child_of(const LevelNode& nd, int c, const uint32_t* rs, const uint8_t* rdesc) {
    Child ch;
    uint32_t a = nd.b[c], b = nd.b[c + 1];
    ch.base = rs[a];
    ch.len = rs[b] - ch.base;
    ch.leaf = (b == a + 1);
    ch.rev = ch.leaf ? rdesc[a] : 0u;
    return ch;
}

template <typename K>
__device__ __forceinline__ K child_get(const Child& ch, const K* leaf, const K* inner, uint32_t pos) {
    if (ch.leaf) return ch.rev ? leaf[ch.base + ch.len - 1 - pos] : leaf[ch.base + pos];
    return inner[ch.base + pos];
}

__global__ void __launch_bounds__(1024) k_level_prep(LevelNode* __restrict__ nodes, uint32_t nn, const uint32_t* __restrict__ rs,
                                                     uint32_t ts, uint64_t* __restrict__ ctr) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
    uint32_t per = (nn + 1023) / 1024;
    uint32_t b = min(nn, threadIdx.x * per), e = min(nn, b + per);
    uint32_t acc = 0;
    for (uint32_t v = b; v < e; v++) {
        const LevelNode& nd = nodes[v];
        uint32_t s = 0;
        for (int c = 0; c < nd.degree; c++) {
            uint32_t len = rs[nd.b[c + 1]] - rs[nd.b[c]];
            uint32_t m = (len + ts - 1) / ts;
            s += m > 0 ? m - 1 : 0;
        }
        acc += s + 1;
    }
    uint32_t tot;
    uint32_t pre = block_sum_excl<1024>(acc, tmp, &tot);
    for (uint32_t v = b; v < e; v++) {
        LevelNode& nd = nodes[v];
        uint32_t s = 0;
        for (int c = 0; c < nd.degree; c++) {
            uint32_t len = rs[nd.b[c + 1]] - rs[nd.b[c]];
            uint32_t m = (len + ts - 1) / ts;
            s += m > 0 ? m - 1 : 0;
        }
        nd.unit_off = pre;
        nd.nunits = s + 1;
        pre += s + 1;
    }
    if (threadIdx.x == 0) ctr[kCtrUnits] = tot;
}

// One block per node: fills unit -> node and the splitter table.  Splitter g
// of the node is element (m+1)*ts of child c; k lanes compute its position in
// every child under the order (key, child, position) and its slot among the
// node's splitters in that order.
template <typename K>
__global__ void __launch_bounds__(256) k_level_split(const LevelNode* __restrict__ nodes, const uint32_t* __restrict__ rs,
                                                     const uint8_t* __restrict__ rdesc, const K* __restrict__ leaf,
                                                     const K* __restrict__ buf0, const K* __restrict__ buf1, uint32_t ts, int k,
                                                     uint32_t* __restrict__ unit_node, uint32_t* __restrict__ tab) {
    const LevelNode nd = nodes[blockIdx.x];
    const int d = nd.degree;
    const K* inner = ((nd.depth + 1) & 1) ? buf1 : buf0;
    for (uint32_t u = threadIdx.x; u < nd.nunits; u += blockDim.x) unit_node[nd.unit_off + u] = blockIdx.x;
    Child ch[8];
    uint32_t cnt[8];
    uint32_t nsplit = 0;
    for (int c = 0; c < d; c++) {
        ch[c] = child_of(nd, c, rs, rdesc);
        uint32_t m = (ch[c].len + ts - 1) / ts;
        cnt[c] = m > 0 ? m - 1 : 0;
        nsplit += cnt[c];
    }
    const uint32_t groups = blockDim.x / k;
    const uint32_t my_c = threadIdx.x % k;
    const uint32_t iters = (nsplit + groups - 1) / groups;
    for (uint32_t it = 0; it < iters; it++) {
        uint32_t g = it * groups + threadIdx.x / k;
        bool active = g < nsplit;
        uint32_t split = 0;
        if (active) {
            uint32_t c = 0, gg = g;
            while (gg >= cnt[c]) { gg -= cnt[c]; c++; }
            uint32_t q = (gg + 1) * ts;
            K key = child_get(ch[c], leaf, inner, q);
            if ((int)my_c < d) {
                if (my_c == c) {
                    split = q;
                } else {
                    const Child& o = ch[my_c];
                    uint32_t lo = 0, hi = o.len;
                    bool upper = my_c < c;  // earlier children win ties: count keys <= key
                    while (lo < hi) {
                        uint32_t mid = (lo + hi) >> 1;
                        K x = child_get(o, leaf, inner, mid);
                        bool before = upper ? (x <= key) : (x < key);
                        if (before) lo = mid + 1; else hi = mid;
                    }
                    split = lo;
                }
            }
        }
        uint32_t m = split ? (split + ts - 1) / ts - 1 : 0u;
        uint32_t slot = m;
        for (int o = 1; o < k; o <<= 1) slot += __shfl_xor_sync(0xffffffffu, slot, o);
        if (active && (int)my_c < d) tab[(size_t)(nd.unit_off + slot + 1) * k + my_c] = split;
    }
}

template <typename K, bool V>
__global__ void __launch_bounds__(kMergeThreads)
    k_level_merge(const LevelNode* __restrict__ nodes, const uint32_t* __restrict__ unit_node, const uint32_t* __restrict__ tab,
                  const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs, const uint8_t* __restrict__ rdesc,
                  const K* __restrict__ leaf, const uint32_t* __restrict__ vleaf, K* __restrict__ buf0, K* __restrict__ buf1,
                  uint32_t* __restrict__ vbuf0, uint32_t* __restrict__ vbuf1, uint32_t C, int k, uint32_t* __restrict__ status) {
    extern __shared__ uint4 smem_raw[];
    K* kA = reinterpret_cast<K*>(smem_raw);
    K* kB = kA + C;
    uint32_t* vA = V ? reinterpret_cast<uint32_t*>(kB + C) : nullptr;
    uint32_t* vB = V ? vA + C : nullptr;
    __shared__ uint32_t st_c[8], off_c[9];
    __shared__ uint16_t seg_start[10], seg_mid[9];
    __shared__ uint32_t sh_ns;
    __shared__ Child chs[8];

    const uint32_t u = blockIdx.x;
    if (u >= (uint32_t)ctr[kCtrUnits]) return;
    const LevelNode nd = nodes[unit_node[u]];
    const int d = nd.degree;
    const uint32_t local = u - nd.unit_off;
    const bool depth_odd = nd.depth & 1;
    const K* inner = depth_odd ? buf0 : buf1;               // children sit at depth + 1
    const uint32_t* vinner = depth_odd ? vbuf0 : vbuf1;
    K* out = depth_odd ? buf1 : buf0;
    uint32_t* vout = depth_odd ? vbuf1 : vbuf0;

    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int c = 0; c < d; c++) {
            Child ch = child_of(nd, c, rs, rdesc);
            chs[c] = ch;
            uint32_t s = local == 0 ? 0u : tab[(size_t)(nd.unit_off + local) * k + c];
            uint32_t e = local + 1 == nd.nunits ? ch.len : tab[(size_t)(nd.unit_off + local + 1) * k + c];
            st_c[c] = s;
            off_c[c] = acc;
            acc += e - s;
        }
        off_c[d] = acc;
    }
    __syncthreads();
    const uint32_t total = off_c[d];
    if (total > C) {
        if (threadIdx.x == 0) dev_fail(status, kDevRange);
        return;
    }
    uint32_t out_base = nd.sL;
    for (int c = 0; c < d; c++) out_base += st_c[c];
    for (int c = 0; c < d; c++) {
        const Child ch = chs[c];
        const uint32_t s = st_c[c], o = off_c[c], m = off_c[c + 1] - o;
        for (uint32_t i = threadIdx.x; i < m; i += kMergeThreads) {
            uint32_t pos = s + i;
            uint32_t src = ch.leaf ? (ch.rev ? ch.base + ch.len - 1 - pos : ch.base + pos) : ch.base + pos;
            kA[o + i] = ch.leaf ? leaf[src] : inner[src];
            if (V) vA[o + i] = ch.leaf ? vleaf[src] : vinner[src];
        }
    }
    __syncthreads();
    K* cur = kA;
    K* oth = kB;
    uint32_t* vcur = vA;
    uint32_t* voth = vB;
    for (uint32_t t = 0; (1 << t) < d; t++) {
        if (threadIdx.x == 0) {
            uint32_t ns = 0;
            seg_start[0] = 0;
            seg_mid[0] = (uint16_t)kNoMid;
            for (int c = 1; c < d; c++) {
                uint32_t cz = __ffs(c) - 1;
                if (cz > t) {
                    ns++;
                    seg_start[ns] = (uint16_t)off_c[c];
                    seg_mid[ns] = (uint16_t)kNoMid;
                } else if (cz == t) {
                    seg_mid[ns] = (uint16_t)off_c[c];
                }
            }
            ns++;
            seg_start[ns] = (uint16_t)total;
            sh_ns = ns;
        }
        __syncthreads();
        merge_pass<K, V>(cur, oth, vcur, voth, total, seg_start, seg_mid, sh_ns);
        __syncthreads();
        K* tk = cur; cur = oth; oth = tk;
        uint32_t* tv = vcur; vcur = voth; voth = tv;
    }
    for (uint32_t i = threadIdx.x; i < total; i += kMergeThreads) {
        out[out_base + i] = cur[i];
        if (V) vout[out_base + i] = vcur[i];
    }
}

template <typename K, bool V>
__global__ void k_copy_single_run(const K* __restrict__ in, const uint32_t* __restrict__ vin, K* __restrict__ out,
                                  uint32_t* __restrict__ vout, uint64_t n, const uint8_t* __restrict__ rdesc) {
    const bool rev = rdesc[0] != 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = rev ? n - 1 - i : i;
        out[i] = in[s];
        if (V) vout[i] = vin[s];
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

MergeGeom merge_geom(int key_bytes, bool vals, int k) {
    MergeGeom g;
    if (key_bytes == 4 && !vals) { g.c_fused = 16384; g.tfix = 4096; g.c_level = 8192; }
    else if (key_bytes == 8 && vals) { g.c_fused = 6144; g.tfix = 1536; g.c_level = 4096; }
    else { g.c_fused = 8192; g.tfix = 2048; g.c_level = 4096; }
    g.tmax = g.c_fused - g.tfix;
    g.k = k;
    g.ts = g.c_level / (uint32_t)k;
    return g;
}

template <typename K, bool V>
void launch_fused(const K* leaf_keys, const uint32_t* leaf_vals, K* out, uint32_t* vout, uint64_t n, const MergeGeom& g,
                  const WsView& ws, cudaStream_t st) {
    size_t smem = SmemLayout<K, V>::bytes(g.c_fused);
    cudaFuncSetAttribute(k_fused<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint32_t grid = ws.windows - 1;
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    k_fused<K, V><<<grid, kMergeThreads, smem, st>>>(leaf_keys, leaf_vals, out, tmp, vout, ws.vals_tmp, ws.run_starts,
                                                     ws.run_desc, ws.powers, ws.fr_end, ws.fr_depth, ws.first_run,
                                                     g.c_fused, g.k, reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus));
    g_launches += 1;
    (void)n;
}

template <typename K>
void launch_level_plan(uint32_t level_off, uint32_t nnodes, int k, const K* leaf_keys, K* out, const MergeGeom& g,
                       const WsView& ws, cudaStream_t st) {
    LevelNode* nodes = ws.nodes_lvl + level_off;
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    k_level_prep<<<1, 1024, 0, st>>>(nodes, nnodes, ws.run_starts, g.ts, ws.counters);
    k_level_split<K><<<nnodes, 256, 0, st>>>(nodes, ws.run_starts, ws.run_desc, leaf_keys, out, tmp, g.ts, k,
                                              ws.unit_node, ws.split_tab);
    g_launches += 2;
}

template <typename K, bool V>
void launch_level_merge(uint32_t level_off, uint32_t nnodes, uint64_t level_elems, int k, const K* leaf_keys,
                        const uint32_t* leaf_vals, K* out, uint32_t* vout, const MergeGeom& g, const WsView& ws,
                        cudaStream_t st) {
    LevelNode* nodes = ws.nodes_lvl + level_off;
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    size_t smem = (size_t)2 * g.c_level * (sizeof(K) + (V ? 4 : 0));
    cudaFuncSetAttribute(k_level_merge<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint64_t bound = level_elems / g.ts + nnodes + 1;
    k_level_merge<K, V><<<(uint32_t)bound, kMergeThreads, smem, st>>>(
        nodes, ws.unit_node, ws.split_tab, ws.counters, ws.run_starts, ws.run_desc, leaf_keys, leaf_vals, out, tmp, vout,
        ws.vals_tmp, g.c_level, k, reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus));
    g_launches += 1;
}

template <typename K, bool V>
void launch_copy_single_run(const K* in, const uint32_t* vin, K* out, uint32_t* vout, uint64_t n, const WsView& ws,
                            cudaStream_t st) {
    uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(n, 256), 152 * 8);
    k_copy_single_run<K, V><<<grid, 256, 0, st>>>(in, vin, out, vout, n, ws.run_desc);
    g_launches += 1;
}

#define MPS_INST(K, V)                                                                                                  \
    template void launch_fused<K, V>(const K*, const uint32_t*, K*, uint32_t*, uint64_t, const MergeGeom&,             \
                                     const WsView&, cudaStream_t);                                                      \
    template void launch_level_merge<K, V>(uint32_t, uint32_t, uint64_t, int, const K*, const uint32_t*, K*, uint32_t*, \
                                           const MergeGeom&, const WsView&, cudaStream_t);                              \
    template void launch_copy_single_run<K, V>(const K*, const uint32_t*, K*, uint32_t*, uint64_t, const WsView&,      \
                                               cudaStream_t);
MPS_INST(uint32_t, false)
MPS_INST(uint32_t, true)
MPS_INST(uint64_t, false)
MPS_INST(uint64_t, true)
#undef MPS_INST
template void launch_level_plan<uint32_t>(uint32_t, uint32_t, int, const uint32_t*, uint32_t*, const MergeGeom&,
                                          const WsView&, cudaStream_t);
template void launch_level_plan<uint64_t>(uint32_t, uint32_t, int, const uint64_t*, uint64_t*, const MergeGeom&,
                                          const WsView&, cudaStream_t);

}  // namespace mps
