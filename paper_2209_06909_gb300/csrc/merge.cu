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

// ---- asynchronous global -> shared copies (cp.async)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (BYTES == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else if (BYTES == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- bulk global -> shared copies on the TMA engine, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Orders this thread's earlier shared-memory accesses before later writes by
// the async (TMA) proxy.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// bytes (a multiple of 16) from 16-byte aligned gmem to 16-byte aligned smem
__device__ __forceinline__ void bulk_copy_g2s(void* smem, const void* gmem, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(smem)),
                 "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
constexpr uint32_t kMbarSpinLimit = 1u << 24;

constexpr int kFusedThreads = 256;
constexpr uint32_t kFusedPad = 16;  // elements of slack per fused-kernel buffer
constexpr uint32_t kNoMid = 0xFFFFu;

// Number of elements of A[0..na) among the first `diag` outputs of the stable
// merge of A and B[0..nb) (A first on equal keys): merge path.
template <typename K>
__device__ __forceinline__ uint32_t merge_path2(const K* __restrict__ A, uint32_t na, const K* __restrict__ B, uint32_t nb,
                                                uint32_t diag) {
    uint32_t l = diag > nb ? diag - nb : 0u, h = min(diag, na);
    while (l < h) {
        const uint32_t mid = (l + h) >> 1;
        if (A[mid] <= B[diag - 1 - mid]) l = mid + 1; else h = mid;
    }
    return l;
}

// Writes outputs [o, stop) of the stable merge of A[ia..na) and B[ib..nb)
// (ties to A).  Every step loads the next element of the side it took, under
// a predicate (one shared-memory load per output).  A[na] and B[nb] are read
// (never used), so one element past each side must be readable shared memory.
template <typename K, bool V>
__device__ __forceinline__ void serial_merge2(const K* __restrict__ A, uint32_t na, const K* __restrict__ B, uint32_t nb,
                                              const uint32_t* __restrict__ vA, const uint32_t* __restrict__ vB,
                                              K* __restrict__ dst, uint32_t* __restrict__ vdst, uint32_t ia, uint32_t ib,
                                              uint32_t o, uint32_t stop) {
    K ka = A[ia];
    K kb = B[ib];
    for (; o < stop; o++) {
        const bool take_a = (ib >= nb) | ((ia < na) & (ka <= kb));
        dst[o] = take_a ? ka : kb;
        if (V) vdst[o] = take_a ? vA[ia] : vB[ib];
        if (take_a) {
            ++ia;
            ka = A[ia];
        } else {
            ++ib;
            kb = B[ib];
        }
    }
}

// The same on one buffer: A = src[s..m), B = src[m..e).
template <typename K>
__device__ __forceinline__ uint32_t merge_path(const K* __restrict__ src, uint32_t s, uint32_t m, uint32_t e, uint32_t diag) {
    return merge_path2(src + s, m - s, src + m, e - m, diag);
}
template <typename K, bool V>
__device__ __forceinline__ void serial_merge(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
                                             uint32_t* __restrict__ vdst, uint32_t ia, uint32_t m, uint32_t ib, uint32_t e,
                                             uint32_t o, uint32_t stop) {
    // positions relative to A = src[.., m) and B = src[m, e): A starts where the merge's A begins (ia is absolute)
    serial_merge2<K, V>(src, m, src + m, e - m, vsrc, V ? vsrc + m : nullptr, dst, vdst, ia, ib - m, o, stop);
}

// Outputs per thread when NT threads share a merge pass of `total` outputs:
// one chunk each, rounded up to an odd count so that the lanes of a warp,
// walking their outputs in step, touch 32 different shared-memory banks.
template <int NT>
__device__ __forceinline__ uint32_t chunk_per_thread(uint32_t total) {
    return ((total + NT - 1) / NT) | 1u;
}

// Entry of the shared-memory boundary list: bits 0..15 element offset,
// 16..23 power, 24..31 the tournament round in which its two sides meet.
__device__ __forceinline__ uint32_t be_off(uint32_t e) { return e & 0xFFFFu; }
__device__ __forceinline__ uint32_t be_pow(uint32_t e) { return (e >> 16) & 0xFFu; }
__device__ __forceinline__ uint32_t be_rnd(uint32_t e) { return e >> 24; }

// Round t of the current level over [0, len), read straight from the sorted
// boundary list bl[0..na): entries with round < t lie inside runs merged by
// earlier rounds, an entry with round t is the midpoint of a merge, and an
// entry with a later round delimits segments.  Between two delimiters there
// is at most one midpoint (the tournament brackets of a node), so the segment
// holding output o is found by a binary search for o and a walk over at most
// 2^t - 1 skipped entries on either side; a segment without a midpoint is
// copied.
// Index of the first boundary-list entry with an offset above this thread's
// first output of a merge round (the same for every round of a level).
__device__ __forceinline__ int round_entry(uint32_t len, const uint32_t* __restrict__ bl, int na) {
    const uint32_t o = threadIdx.x * chunk_per_thread<kFusedThreads>(len);
    int lo = 0, hi = na;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (be_off(bl[mid]) <= o) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename K, bool V>
__device__ __forceinline__ void merge_round(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
                                            uint32_t* __restrict__ vdst, uint32_t len, const uint32_t* __restrict__ bl,
                                            int na, int first, uint32_t t) {
    const uint32_t ipt = chunk_per_thread<kFusedThreads>(len);
    const uint32_t base = threadIdx.x * ipt;
    if (base >= len) return;
    uint32_t o = base;
    const uint32_t oe = min(base + ipt, len);
    int j = first - 1;  // nearest entry at or left of o that this round sees (-1: the start)
    while (j >= 0 && be_rnd(bl[j]) < t) j--;
    while (o < oe) {
        int nx = j + 1;
        while (nx < na && be_rnd(bl[nx]) < t) nx++;
        uint32_t s, m = kNoMid, e;
        if (j >= 0 && be_rnd(bl[j]) == t) {
            // o lies in the right half of a merge whose left delimiter precedes j
            m = be_off(bl[j]);
            int jl = j - 1;
            while (jl >= 0 && be_rnd(bl[jl]) < t) jl--;
            s = jl >= 0 ? be_off(bl[jl]) : 0u;
            e = nx < na ? be_off(bl[nx]) : len;
            j = nx;
        } else {
            s = j >= 0 ? be_off(bl[j]) : 0u;
            if (nx < na && be_rnd(bl[nx]) == t) {
                m = be_off(bl[nx]);
                int n2 = nx + 1;
                while (n2 < na && be_rnd(bl[n2]) < t) n2++;
                e = n2 < na ? be_off(bl[n2]) : len;
                j = n2;
            } else {
                e = nx < na ? be_off(bl[nx]) : len;
                j = nx;
            }
        }
        const uint32_t stop = min(e, oe);
        if (m == kNoMid || m >= e || m <= s) {
            for (; o < stop; o++) {
                dst[o] = src[o];
                if (V) vdst[o] = vsrc[o];
            }
        } else {
            const uint32_t l = merge_path(src, s, m, e, o - s);
            serial_merge<K, V>(src, dst, vsrc, vdst, s + l, m, m + (o - s) - l, e, o, stop);
            o = stop;
        }
    }
}

// Items per thread for a blocked loop over m items: ceil(m / threads), rounded
// up to an odd number (conflict-free shared-memory strides).
__device__ __forceinline__ uint32_t odd_chunk(uint32_t m) {
    uint32_t per = (m + kFusedThreads - 1) / kFusedThreads;
    return per | 1u;
}

// (count in bits 0..31, summed; bit set in bits 32..63, OR-ed)
struct OpSumOr {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const {
        return (((a & 0xFFFFFFFFull) + (b & 0xFFFFFFFFull)) & 0xFFFFFFFFull) | ((a | b) & 0xFFFFFFFF00000000ull);
    }
};

struct OpMax2 {
    __device__ uint4 operator()(uint4 X, uint4 Y) const { return make_uint4(max(X.x, Y.x), max(X.y, Y.y), 0u, 0u); }
};

template <typename K, bool V>
struct FusedSmem {
    // key and payload buffers of C elements plus kFusedPad of slack (the loaded
    // tile sits on its source's 16-byte grid; merges read two past the end)
    static __host__ __device__ size_t bytes(uint32_t C) {
        const uint32_t bmax = C / 2 + 8;
        const size_t cp = (size_t)C + kFusedPad;
        return 2 * cp * sizeof(K) + (V ? 2 * cp * 4 : 0) + (size_t)2 * bmax * 4;
    }
};

// Fused subtrees: persistent blocks over the list of fused tiles of at most C
// elements: a maximal subtree, or consecutive sibling subtrees together with
// their parent's power as a floor (levels at or below the floor are not merged
// here, so the siblings stay apart).  A block loads one tile (reversing
// strictly descending runs), executes all its levels in shared memory, largest
// power first, and writes the result.  Level p: the boundaries of power p form
// groups between boundaries of smaller power (one group = one node); the
// group index q of each boundary gives the tournament round ctz(q) in which
// its two sides meet.
template <typename K, bool V>
__global__ void __launch_bounds__(kFusedThreads)
    k_fused(const uint4* __restrict__ flist, const uint64_t* __restrict__ ctr, const K* __restrict__ leaf,
            const uint32_t* __restrict__ vleaf, K* __restrict__ out0, K* __restrict__ out1, uint32_t* __restrict__ vout0,
            uint32_t* __restrict__ vout1, const uint32_t* __restrict__ rs, const uint8_t* __restrict__ rdesc,
            const uint8_t* __restrict__ P, uint32_t C, int k, uint64_t n_total, uint32_t* __restrict__ status,
            unsigned long long* __restrict__ next_tile) {
    extern __shared__ uint4 smem_raw[];
    const uint32_t BMAX = C / 2 + 8;
    const uint32_t CP = C + kFusedPad;
    K* kA = reinterpret_cast<K*>(smem_raw);
    K* kB = kA + CP;
    uint32_t* vA = V ? reinterpret_cast<uint32_t*>(kB + CP) : nullptr;
    uint32_t* vB = V ? vA + CP : nullptr;
    uint32_t* bl0 = V ? (vB + CP) : reinterpret_cast<uint32_t*>(kB + CP);
    uint32_t* bl1 = bl0 + BMAX;
    __shared__ unsigned long long stmp8[kFusedThreads / 32 + 1];
    __shared__ uint4 stmp4[kFusedThreads / 32 + 1];
    __shared__ __align__(8) uint64_t s_bar;
    // strictly descending runs longer than kShortRun, reversed by the whole block
    constexpr uint32_t kShortRun = 64, kMaxLongRuns = 96;
    __shared__ uint32_t s_long[kMaxLongRuns];
    __shared__ uint32_t s_nlong;
    uint32_t phase = 0;
    const uint32_t tid = threadIdx.x;
    const uint32_t F = (uint32_t)ctr[kCtrFrontier];
    if (tid == 0) mbar_init(&s_bar, 1);
    __syncthreads();

    // tiles are taken one at a time from a counter (their sizes differ, so a
    // fixed assignment would leave some blocks working long after the others)
    __shared__ uint32_t s_f;
    for (;;) {
        __syncthreads();  // every thread has read the previous tile index
        if (tid == 0) s_f = (uint32_t)atomicAdd(next_tile, 1ull);
        __syncthreads();
        const uint32_t f = s_f;
        if (f >= F) break;
        const uint4 fr = flist[f];
        const uint32_t L = fr.x, R = fr.y;
        const bool odd = fr.z & 1u;
        if (tid == 0) s_nlong = 0;
        const uint32_t floor_p = fr.w;  // boundaries of power <= floor_p are never merged here
        if (L >= R) {
            if (tid == 0) dev_fail(status, kDevFusedRange);
            continue;
        }
        const uint32_t s_lo = rs[L];
        const uint32_t len = rs[R] - s_lo;
        if (len > C) {
            if (tid == 0) dev_fail(status, kDevRange);
            return;
        }
        if ((uint64_t)s_lo + len > n_total) {
            if (tid == 0) dev_fail(status, kDevFusedRange);
            continue;
        }
        const uint32_t nruns = R - L;
        const uint32_t nb = nruns - 1;

        // ---- load boundaries, keys and run directions (asynchronous copies)
        // run starts -> kB (as u32), powers and directions -> bl1 (bytes, from
        // 4-byte aligned supersets; both arrays are padded past r)
        uint32_t* rsS = reinterpret_cast<uint32_t*>(kB);
        uint8_t* PS = reinterpret_cast<uint8_t*>(bl1);
        uint8_t* dflag = PS + (C / 2 + 64);
        const uint32_t pa = (L + 1) & ~3u, pb = (R + 3) & ~3u;
        const uint32_t da = L & ~3u, db = (R + 3) & ~3u;
        // keys: element x lands at kA[lead + x], on the 16-byte grid of its
        // source, so the aligned middle is one bulk copy (TMA) completed on
        // s_bar; the unaligned ends and the payloads are copied per element
        constexpr uint32_t VK = 16 / sizeof(K);
        const K* ksrc = leaf + s_lo;
        const uint32_t lead = (uint32_t)((reinterpret_cast<uintptr_t>(ksrc) & 15u) / sizeof(K));
        const uint32_t kib = min(len, (VK - lead) & (VK - 1u));
        const uint32_t kie = kib + (len - kib) / VK * VK;
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, (kie - kib) * (uint32_t)sizeof(K));
            if (kie > kib) bulk_copy_g2s(kA + lead + kib, ksrc + kib, (kie - kib) * (uint32_t)sizeof(K), &s_bar);
        }
        for (uint32_t e = tid; e < nb; e += kFusedThreads) cp_async<4>(rsS + e, rs + L + 1 + e);
        for (uint32_t q = pa + 4 * tid; q < pb; q += 4 * kFusedThreads) cp_async<4>(PS + (q - pa), P + q);
        for (uint32_t q = da + 4 * tid; q < db; q += 4 * kFusedThreads) cp_async<4>(dflag + (q - da), rdesc + q);
        for (uint32_t x = tid; x < kib; x += kFusedThreads) cp_async<sizeof(K)>(kA + lead + x, ksrc + x);
        for (uint32_t x = kie + tid; x < len; x += kFusedThreads) cp_async<sizeof(K)>(kA + lead + x, ksrc + x);
        if (V)
            for (uint32_t x = tid; x < len; x += kFusedThreads) cp_async<4>(vA + lead + x, vleaf + s_lo + x);
        cp_async_commit();
        cp_async_wait<0>();
        {
            uint32_t spins = 0;
            bool done = mbar_try_wait(&s_bar, phase);
            while (!done && spins < kMbarSpinLimit) {
                done = mbar_try_wait(&s_bar, phase);
                spins++;
            }
            if (__syncthreads_or(!done)) {
                // The bulk copy did not complete: report it, one more bounded wait, stop.
                // The copy is well formed by construction (16-byte aligned source and
                // destination, a size that is a multiple of 16 inside the tile's buffer,
                // the expected byte count set before it is issued), so it completes
                // unless the memory system fails; this branch only keeps that case from
                // hanging the GPU, and the status tells the host the output is invalid.
                if (tid == 0) dev_fail(status, kDevSpin);
                for (spins = 0; !mbar_try_wait(&s_bar, phase) && spins < kMbarSpinLimit; spins++) {
                }
                return;
            }
            phase ^= 1u;
        }
        for (uint32_t e = tid; e < nb; e += kFusedThreads)
            bl0[e] = (rsS[e] - s_lo) | ((uint32_t)PS[e + (L + 1 - pa)] << 16);
        dflag += L - da;  // dflag[q] = direction of run L + q
        __syncthreads();

        // ---- reverse the strictly descending runs in place (kA, from lead on):
        // each thread swaps the short runs among its own, the block the long ones
        K* tile = kA + lead;
        uint32_t* vtile = V ? vA + lead : nullptr;
        {
            const uint32_t per_r = odd_chunk(nruns);
            const uint32_t r0 = min(nruns, tid * per_r), r1 = min(nruns, r0 + per_r);
            for (uint32_t r = r0; r < r1; r++) {
                if (!dflag[r]) continue;
                const uint32_t a = r ? be_off(bl0[r - 1]) : 0u;
                const uint32_t b = r + 1 < nruns ? be_off(bl0[r]) : len;
                if (b - a > kShortRun) {
                    const uint32_t slot = atomicAdd(&s_nlong, 1u);
                    if (slot < kMaxLongRuns) s_long[slot] = r;
                    continue;
                }
                for (uint32_t x = a, y = b - 1; x < y; x++, y--) {
                    const K t0 = tile[x];
                    tile[x] = tile[y];
                    tile[y] = t0;
                    if (V) {
                        const uint32_t u0 = vtile[x];
                        vtile[x] = vtile[y];
                        vtile[y] = u0;
                    }
                }
            }
            __syncthreads();
            // a run longer than kShortRun of at most C elements: fewer than kMaxLongRuns
            const uint32_t nlong = min(s_nlong, kMaxLongRuns);
            for (uint32_t j = 0; j < nlong; j++) {
                const uint32_t r = s_long[j];
                const uint32_t a = r ? be_off(bl0[r - 1]) : 0u;
                const uint32_t b = r + 1 < nruns ? be_off(bl0[r]) : len;
                for (uint32_t x = a + tid; x < a + (b - a) / 2; x += kFusedThreads) {
                    const uint32_t y = a + b - 1 - x;
                    const K t0 = tile[x];
                    tile[x] = tile[y];
                    tile[y] = t0;
                    if (V) {
                        const uint32_t u0 = vtile[x];
                        vtile[x] = vtile[y];
                        vtile[y] = u0;
                    }
                }
            }
        }

        // ---- range of powers in the subtree
        uint32_t per = odd_chunk(nb);
        uint32_t e0 = min(nb, tid * per), e1 = min(nb, e0 + per);
        uint32_t pmax, pmin;
        {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            for (uint32_t e = e0; e < e1; e++) {
                const uint32_t p = be_pow(bl0[e]);
                v.x = max(v.x, p);
                v.y = max(v.y, 255u - p);
            }
            const uint4 t = block_reduce<kFusedThreads>(v, OpMax2(), make_uint4(0u, 0u, 0u, 0u), stmp4);
            pmax = t.x;
            pmin = 255u - t.y;
        }
        K* cur = tile;
        K* oth = kB;
        uint32_t* vcur = vtile;
        uint32_t* voth = vB;
        uint32_t na = nb;
        // boundary list of the current level and the list the next level gets
        // (bl1 is free once the load and reversal are done)
        uint32_t* blc = bl0;
        uint32_t* bln = bl1;
        uint32_t T = 0;  // tournament rounds per node: log2 k
        while ((1u << T) < (uint32_t)k) T++;

        for (uint32_t p = pmax; p >= pmin && p >= 1 && p > floor_p; p--) {
            per = odd_chunk(na);
            e0 = min(na, tid * per);
            e1 = min(na, e0 + per);
            // Round of each boundary: for power p, ctz(q) with q its index in the
            // group of power-p boundaries that forms one node (the bracket round
            // of the node's tournament); T for a smaller power (a delimiter).
            // The list holds no power above p any more, so a group's boundaries
            // are adjacent: q is found by looking back at most k - 1 entries.
            uint32_t nk = 0, rmask = 0;
            for (uint32_t e = e0; e < e1; e++) {
                const uint32_t v = blc[e];
                if (be_pow(v) == p) {
                    uint32_t q = 1;
                    while (q < (uint32_t)kMaxFanIn && e >= q && be_pow(blc[e - q]) == p) q++;
                    const uint32_t rd = min((uint32_t)__ffs(q) - 1u, T - 1u);
                    blc[e] = (v & 0x00FFFFFFu) | (rd << 24);
                    rmask |= 1u << rd;
                } else {
                    blc[e] = (v & 0x00FFFFFFu) | (T << 24);
                    nk++;
                }
            }
            // one scan gives each thread's place in the next list, that list's
            // length, and the rounds this level plays
            unsigned long long tot;
            const unsigned long long pre = block_scan_excl<kFusedThreads, false>(
                (unsigned long long)nk | ((unsigned long long)rmask << 32), OpSumOr(), 0ull, stmp8, &tot);
            const uint32_t kpos = (uint32_t)pre, nkeep = (uint32_t)tot;
            if (nkeep == na) continue;  // no boundary of power p in this subtree
            const uint32_t rounds = (uint32_t)(tot >> 32);
            const int first = round_entry(len, blc, (int)na);
            // tournament rounds
            for (uint32_t t = 0; t < T; t++) {
                if (!((rounds >> t) & 1u)) continue;
                merge_round<K, V>(cur, oth, vcur, voth, len, blc, (int)na, first, t);
                __syncthreads();
                K* tk = cur; cur = oth; oth = tk;
                uint32_t* tv = vcur; vcur = voth; voth = tv;
            }
            // the boundaries of smaller power (round tag T) form the next list
            uint32_t w = kpos;
            for (uint32_t e = e0; e < e1; e++) {
                const uint32_t v = blc[e];
                if (be_rnd(v) == T) bln[w++] = v & 0x00FFFFFFu;
            }
            uint32_t* tb = blc; blc = bln; bln = tb;
            na = nkeep;
            __syncthreads();
        }

        // ---- the subtree's output
        K* o = odd ? out1 : out0;
        uint32_t* vo = odd ? vout1 : vout0;
        for (uint32_t x = tid; x < len; x += kFusedThreads) {
            o[s_lo + x] = cur[x];
            if (V) vo[s_lo + x] = vcur[x];
        }
        __syncthreads();
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

__device__ __forceinline__ uint32_t node_splitters(const LevelNode& nd, const uint32_t* rs, uint32_t ts) {
    uint32_t s = 0;
    for (int c = 0; c < nd.degree; c++) {
        uint32_t len = rs[nd.b[c + 1]] - rs[nd.b[c]];
        uint32_t m = (len + ts - 1) / ts;
        s += m > 0 ? m - 1 : 0;
    }
    return s;
}

// Splitters of every node of the level (one thread per node), kept in nsplit.
__global__ void __launch_bounds__(256) k_level_count(LevelNode* __restrict__ nodes_lvl, const uint32_t* __restrict__ level_off,
                                                     int p, const uint32_t* __restrict__ rs, uint32_t ts,
                                                     const uint64_t* __restrict__ ctr) {
    LevelNode* nodes = nodes_lvl + level_off[p];
    const uint32_t nn = (uint32_t)ctr[kCtrHbmCount + p];
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x)
        nodes[v].nsplit = node_splitters(nodes[v], rs, ts);
}

// Per node of the level: offsets of its splitters and work units (one unit
// more than splitters), and unit_node for each node's first unit.
__global__ void __launch_bounds__(1024) k_level_prep(LevelNode* __restrict__ nodes_lvl, const uint32_t* __restrict__ level_off,
                                                     int p, uint64_t* __restrict__ ctr, uint32_t* __restrict__ unit_node) {
    LevelNode* nodes = nodes_lvl + level_off[p];
    const uint32_t nn = (uint32_t)ctr[kCtrHbmCount + p];
    __shared__ uint32_t tmp[1024 / 32 + 1];
    uint32_t per = (nn + 1023) / 1024;
    uint32_t b = min(nn, threadIdx.x * per), e = min(nn, b + per);
    uint32_t acc = 0;
    for (uint32_t v = b; v < e; v++) acc += nodes[v].nsplit;
    uint32_t tot;
    uint32_t pre = block_sum_excl<1024>(acc, tmp, &tot);
    for (uint32_t v = b; v < e; v++) {
        LevelNode& nd = nodes[v];
        const uint32_t s = nd.nsplit;
        nd.split_off = pre;
        nd.nsplit = s;
        nd.unit_off = pre + v;   // units of node v: splitters before it plus one per earlier node
        nd.nunits = s + 1;
        unit_node[pre + v] = v;
        pre += s;
    }
    if (threadIdx.x == 0) {
        ctr[kCtrSplits] = tot;
        ctr[kCtrIntervals] = tot + nn;
    }
}

// Number of elements of child o that come before `key` (<= key if upper,
// else < key): the first position whose element does not.  The child is
// sorted, so the answer is found by narrowing [l, h] with the known elements
// A[l] (before) and A[h] (not before): each step probes the position that
// interpolation between their keys predicts, and adds a bisection probe when
// that did not at least halve the range, so it never takes more than twice
// the probes of a binary search and few on evenly spread keys.  These are
// dependent global loads, the cost of this kernel.
template <typename K>
__device__ __forceinline__ uint32_t count_before(const Child& o, const K* leaf, const K* inner, K key, bool upper) {
    if (o.len == 0) return 0u;
    uint32_t l = 0, h = o.len - 1;
    const K a = child_get(o, leaf, inner, l), b = child_get(o, leaf, inner, h);
    if (!(upper ? (a <= key) : (a < key))) return 0u;
    if (upper ? (b <= key) : (b < key)) return o.len;
    K kl = a, kh = b;  // kl before, kh not before, so kl <= key <= kh and kl < kh
    while (h - l > 1) {
        const uint32_t span = h - l;
        const float f = (float)(key - kl) / (float)(kh - kl);
        uint32_t g = l + 1u + (uint32_t)(f * (float)(span - 1u));
        g = min(max(g, l + 1u), h - 1u);
        K x = child_get(o, leaf, inner, g);
        if (upper ? (x <= key) : (x < key)) { l = g; kl = x; } else { h = g; kh = x; }
        if (2u * (h - l) > span && h - l > 1) {
            const uint32_t mid = l + ((h - l) >> 1);
            x = child_get(o, leaf, inner, mid);
            if (upper ? (x <= key) : (x < key)) { l = mid; kl = x; } else { h = mid; kh = x; }
        }
    }
    return h;
}

// k lanes per splitter, all splitters of the level across the grid.  Splitter
// g of node v is element (m+1)*ts of child c; lane c' finds its position in
// child c' under the order (key, child, position); the k positions give the
// splitter's slot among the node's splitters, i.e. the work unit it starts.
template <typename K>
__global__ void __launch_bounds__(256) k_level_split(const LevelNode* __restrict__ nodes_lvl,
                                                     const uint32_t* __restrict__ level_off, int p,
                                                     const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs,
                                                     const uint8_t* __restrict__ rdesc, const K* __restrict__ leaf,
                                                     const K* __restrict__ buf0, const K* __restrict__ buf1, uint32_t ts, int k,
                                                     uint32_t* __restrict__ unit_node, uint32_t* __restrict__ tab) {
    const LevelNode* nodes = nodes_lvl + level_off[p];
    const uint32_t nn = (uint32_t)ctr[kCtrHbmCount + p];
    const uint32_t total = (uint32_t)ctr[kCtrSplits];
    uint32_t* status = reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(ctr) + kCtrStatus);
    const uint32_t my_c = threadIdx.x % k;
    // grid-stride over splitters; the k lanes of a splitter stay in one warp
    const uint32_t groups_per_grid = gridDim.x * (blockDim.x / k);
    const uint32_t iters = (total + groups_per_grid - 1) / groups_per_grid;
    for (uint32_t it = 0; it < iters; it++) {
    const uint32_t g = it * groups_per_grid + blockIdx.x * (blockDim.x / k) + threadIdx.x / k;
    const bool active = g < total;
    uint32_t split = 0, v = 0, c = 0, unit_base = 0, nsp = 0;
    int d = 0;
    if (active) {
        // the node holding splitter g: the last node with split_off <= g.  With
        // s_lo = split_off[lo] <= g < s_hi = split_off[hi] (split_off[nn] read as
        // the total), each step probes where interpolation between s_lo and s_hi
        // puts g, and adds a bisection probe when that did not at least halve
        // [lo, hi]; split_off grows with v almost linearly, so a few probes do
        uint32_t lo = 0, hi = nn, s_lo = 0, s_hi = total;
        while (hi - lo > 1) {
            const uint32_t span = hi - lo;
            uint32_t m = lo + (uint32_t)(((uint64_t)(g - s_lo) * span) / (uint64_t)(s_hi - s_lo));
            m = min(max(m, lo + 1u), hi - 1u);
            uint32_t sm = nodes[m].split_off;
            if (sm <= g) { lo = m; s_lo = sm; } else { hi = m; s_hi = sm; }
            if (2u * (hi - lo) > span && hi - lo > 1) {
                m = lo + ((hi - lo) >> 1);
                sm = nodes[m].split_off;
                if (sm <= g) { lo = m; s_lo = sm; } else { hi = m; s_hi = sm; }
            }
        }
        v = lo;
        const LevelNode nd = nodes[v];
        d = nd.degree;
        unit_base = nd.unit_off;
        nsp = nd.nsplit;
        const K* inner = ((nd.depth + 1) & 1) ? buf1 : buf0;
        uint32_t gg = g - nd.split_off;
        Child ch_c;
        for (c = 0; c < (uint32_t)d; c++) {
            ch_c = child_of(nd, c, rs, rdesc);
            uint32_t m = (ch_c.len + ts - 1) / ts;
            uint32_t cnt = m > 0 ? m - 1 : 0;
            if (gg < cnt) break;
            gg -= cnt;
        }
        const uint32_t q = (gg + 1) * ts;
        const K key = child_get(ch_c, leaf, inner, q);
        if ((int)my_c < d) {
            if (my_c == c) {
                split = q;
            } else {
                const Child o = child_of(nd, my_c, rs, rdesc);
                const bool upper = my_c < c;  // earlier children win ties: count keys <= key
                split = count_before(o, leaf, inner, key, upper);
            }
        }
    }
    uint32_t slot = split ? (split + ts - 1) / ts - 1 : 0u;
    for (int o = 1; o < k; o <<= 1) slot += __shfl_xor_sync(0xffffffffu, slot, o);
    // sorted children give every splitter a slot below the node's splitter
    // count; anything else (a child that is not sorted) is reported, not written
    if (active && slot >= nsp) {
        if (my_c == 0) dev_fail(status, kDevSplitSlot);
    } else if (active) {
        if ((int)my_c < d) tab[(size_t)(unit_base + slot + 1) * k + my_c] = split;
        if (my_c == 0) unit_node[unit_base + slot + 1] = v;
    }
    }
}

// One work unit of a level: a contiguous slice of each child of one node
// (192 bytes, read into shared memory one unit ahead).
struct __align__(16) UnitDesc {
    uint32_t out_base;               // first output element
    uint32_t total;                  // elements in the unit
    uint32_t d;                      // bits 0..7: number of children; bit 31: odd depth
    uint32_t flags;                  // bit c: slice c is a leaf; bit 16+c: read backwards
    uint32_t off[kMaxFanIn + 1];     // slice offsets in shared memory (off[d] = total)
    uint32_t src[kMaxFanIn];         // element of the slice's source that lands at off[c]
    uint32_t pad[11];
};
static_assert(sizeof(UnitDesc) == kUnitDescBytes, "UnitDesc layout");
constexpr int kUnitDescVec = (int)(sizeof(UnitDesc) / 16);  // 16-byte words per descriptor

// Splitter intervals are packed into work units greedily: walking a run of
// consecutive intervals, a unit starts at the first interval of a node, at
// the first interval of the run, and at every interval that would take the
// unit past c elements; otherwise the interval joins the open unit.  With
// splitters every ts = c/k elements of each of at most k children no
// interval exceeds c, so every interval fits a unit on its own; intervals
// average ts elements, so a unit usually takes several.  (Measured on the
// 2^28 permutation at k = 4: c/k beats c/(2k), which doubles the splitter
// searches, and 3c/(4k).)  Each thread packs its own run of kPackItems intervals, so
// runs are packed independently (a run boundary always starts a unit).
constexpr int kPackThreads = 128;
constexpr int kPackItems = kPackTile / kPackThreads;
static_assert(kPackItems % 4 == 0, "16-byte loads of interval sizes");

__device__ __forceinline__ uint32_t interval_rank(const uint32_t* __restrict__ tab, uint32_t i, int k, uint32_t d) {
    uint32_t r = 0;
    for (uint32_t c = 0; c < d; c++) r += tab[(size_t)i * k + c];
    return r;
}

// Size of every interval of the level (elements), with bit 31 set on the
// first interval of each node: isz[i] for i < ctr[kCtrIntervals].
__global__ void __launch_bounds__(256) k_interval_size(const LevelNode* __restrict__ nodes_lvl,
                                                       const uint32_t* __restrict__ level_off, int p,
                                                       const uint32_t* __restrict__ unit_node, const uint32_t* __restrict__ tab,
                                                       const uint64_t* __restrict__ ctr, int k, uint32_t* __restrict__ isz) {
    const LevelNode* nodes = nodes_lvl + level_off[p];
    const uint32_t nn = (uint32_t)ctr[kCtrHbmCount + p];
    uint32_t* status = reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(ctr) + kCtrStatus);
    const uint32_t ni = (uint32_t)ctr[kCtrIntervals];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
        const uint32_t v = unit_node[i];
        if (v >= nn) {
            dev_fail(status, kDevPackNode);
            isz[i] = 1u << 31;  // an empty interval that starts a unit
            continue;
        }
        const LevelNode& nd = nodes[v];
        const uint32_t local = i - nd.unit_off;
        const uint32_t r0 = local == 0 ? 0u : interval_rank(tab, i, k, nd.degree);
        const uint32_t r1 = local + 1 < nd.nunits ? interval_rank(tab, i + 1, k, nd.degree) : nd.sR - nd.sL;
        isz[i] = ((r1 - r0) & 0x7FFFFFFFu) | (local == 0 ? 1u << 31 : 0u);
    }
}

// Greedy packing of intervals [i0, i0 + kPackItems) clipped to ni: returns
// the number of units that start there and, if `out` is given, writes the
// index of each starting interval.  isz is padded past ni, so the 16-byte
// loads of the last run stay inside it.
__device__ __forceinline__ uint32_t pack_run(const uint32_t* __restrict__ isz, uint32_t i0, uint32_t ni, uint32_t c,
                                             uint32_t* __restrict__ out) {
    uint32_t cnt = 0, acc = 0;
    const uint4* s4 = reinterpret_cast<const uint4*>(isz + i0);
#pragma unroll 4
    for (uint32_t q = 0; q < (uint32_t)kPackItems / 4; q++) {
        const uint4 w4 = s4[q];
        const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (uint32_t t = 0; t < 4; t++) {
            const uint32_t j = 4 * q + t;
            if (i0 + j < ni) {
                const uint32_t sz = w[t] & 0x7FFFFFFFu;
                if (j == 0 || (w[t] >> 31) || acc + sz > c) {
                    if (out) out[cnt] = i0 + j;
                    cnt++;
                    acc = sz;
                } else {
                    acc += sz;
                }
            }
        }
    }
    return cnt;
}

__global__ void __launch_bounds__(kPackThreads) k_pack_reduce(const uint32_t* __restrict__ isz, const uint64_t* __restrict__ ctr,
                                                              uint32_t c, uint32_t* __restrict__ tiles) {
    __shared__ uint32_t tmp[kPackThreads / 32 + 1];
    const uint32_t ni = (uint32_t)ctr[kCtrIntervals];
    const uint32_t i0 = blockIdx.x * kPackTile + threadIdx.x * kPackItems;
    const uint32_t cnt = i0 < ni ? pack_run(isz, i0, ni, c, nullptr) : 0u;
    uint32_t tot;
    block_sum_excl<kPackThreads>(cnt, tmp, &tot);
    if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_pack_scan(uint32_t* __restrict__ tiles, uint32_t ntiles, uint64_t* __restrict__ ctr) {
    __shared__ uint32_t tmp[1024 / 32 + 1];
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
    if (threadIdx.x == 0) ctr[kCtrUnits] = tot;
}

__global__ void __launch_bounds__(kPackThreads) k_pack_apply(const uint32_t* __restrict__ isz, const uint64_t* __restrict__ ctr,
                                                             uint32_t c, const uint32_t* __restrict__ tiles,
                                                             uint32_t* __restrict__ unit_first) {
    __shared__ uint32_t tmp[kPackThreads / 32 + 1];
    const uint32_t ni = (uint32_t)ctr[kCtrIntervals];
    const uint32_t i0 = blockIdx.x * kPackTile + threadIdx.x * kPackItems;
    const uint32_t cnt = i0 < ni ? pack_run(isz, i0, ni, c, nullptr) : 0u;
    const uint32_t pos = tiles[blockIdx.x] + block_sum_excl<kPackThreads>(cnt, tmp, nullptr);
    if (i0 < ni) pack_run(isz, i0, ni, c, unit_first + pos);
}

// One thread per packed work unit of the level: fills its descriptor.
__global__ void __launch_bounds__(256) k_level_desc(const LevelNode* __restrict__ nodes_lvl, const uint32_t* __restrict__ level_off,
                                                    int p, const uint32_t* __restrict__ unit_node,
                                                    const uint32_t* __restrict__ unit_first, const uint32_t* __restrict__ tab,
                                                    const uint64_t* __restrict__ ctr, const uint32_t* __restrict__ rs,
                                                    const uint8_t* __restrict__ rdesc, int k, UnitDesc* __restrict__ out) {
    const LevelNode* nodes = nodes_lvl + level_off[p];
    const uint32_t nn = (uint32_t)ctr[kCtrHbmCount + p];
    uint32_t* status = reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(ctr) + kCtrStatus);
    const uint32_t nu = (uint32_t)ctr[kCtrUnits];
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    const uint32_t i0 = unit_first[u];
    const uint32_t v = unit_node[i0];
    if (v >= nn) {
        dev_fail(status, kDevUnitNode);
        UnitDesc Z;
        for (int q = 0; q < (int)(sizeof(UnitDesc) / 4); q++) reinterpret_cast<uint32_t*>(&Z)[q] = 0;
        out[u] = Z;
        continue;
    }
    const LevelNode& nd = nodes[v];
    const uint32_t d = nd.degree;
    const uint32_t node_end = nd.unit_off + nd.nunits;   // one past the node's last interval
    uint32_t i1 = node_end;
    if (u + 1 < nu) {
        const uint32_t nx = unit_first[u + 1];
        if (nx < node_end) i1 = nx;
    }
    const bool first = i0 == nd.unit_off, last = i1 == node_end;
    UnitDesc D;
    uint32_t acc = 0, ob = nd.sL, flags = 0;
    for (uint32_t c = 0; c < (uint32_t)kMaxFanIn; c++) {
        if (c < d) {
            const uint32_t a = nd.b[c], b = nd.b[c + 1];
            const uint32_t base = rs[a], len = rs[b] - base;
            const uint32_t st = first ? 0u : tab[(size_t)i0 * k + c];
            const uint32_t en = last ? len : tab[(size_t)i1 * k + c];
            const uint32_t leaf = (b == a + 1);
            const uint32_t rev = leaf ? rdesc[a] : 0u;
            D.src[c] = rev ? base + len - 1 - st : base + st;
            flags |= (leaf << c) | (rev << (16 + c));
            D.off[c] = acc;
            acc += en - st;
            ob += st;
        } else {
            D.src[c] = 0;
            D.off[c] = acc;
        }
    }
    D.off[kMaxFanIn] = acc;
    D.out_base = ob;
    D.total = acc;
    D.d = d | ((nd.depth & 1u) << 31);
    D.flags = flags;
    for (int q = 0; q < 11; q++) D.pad[q] = 0;
    out[u] = D;
    }
}

constexpr int kLvlThreads = 256;
// elements of slack per level-merge buffer: each of up to kMaxFanIn slices
// starts on its source's 16-byte grid and ends rounded up to it (at most 6
// elements of gap per slice for 4-byte keys), plus the output shift
constexpr uint32_t kLvlPad = 128;

// Block-wide copy of src[0..total) (shared memory) to dst[0..total) (global),
// where src + q and dst + q share their offset within 16 bytes (src sits
// `shift` elements past a 16-byte boundary): scalar head and tail, 16-byte
// vectors in between.
template <typename T>
__device__ __forceinline__ void store_vec(T* __restrict__ dst, const T* __restrict__ src, uint32_t total, uint32_t shift) {
    constexpr uint32_t VE = 16 / sizeof(T);
    const uint32_t head = min(total, (VE - shift) & (VE - 1u));
    const uint32_t nvec = (total - head) / VE;
    for (uint32_t q = threadIdx.x; q < head; q += kLvlThreads) dst[q] = src[q];
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    uint4* d4 = reinterpret_cast<uint4*>(dst + head);
    for (uint32_t q = threadIdx.x; q < nvec; q += kLvlThreads) d4[q] = s4[q];
    for (uint32_t q = head + nvec * VE + threadIdx.x; q < total; q += kLvlThreads) dst[q] = src[q];
}

// Round t of the tournament over the unit's d slices: slices are grouped in
// blocks of 2^(t+1); the two halves of every block are merged (stable, left
// first), a block without a right half is copied.
template <typename K, bool V>
__device__ __forceinline__ void unit_round(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
                                           uint32_t* __restrict__ vdst, const uint32_t* __restrict__ off, uint32_t d,
                                           uint32_t t) {
    const uint32_t step = 1u << (t + 1), half = 1u << t;
    const uint32_t total = off[d];
    const uint32_t ipt = chunk_per_thread<kLvlThreads>(total);
    {
        const uint32_t base = threadIdx.x * ipt;
        if (base >= total) return;
        uint32_t o = base;
        const uint32_t oe = min(base + ipt, total);
        uint32_t c0 = 0;
        for (uint32_t c = step; c < d; c += step)
            if (off[c] <= o) c0 = c;
        while (o < oe) {
            const uint32_t cm = c0 + half, c1 = min(c0 + step, d);
            const uint32_t s = off[c0], e = off[c1];
            const uint32_t stop = min(e, oe);
            if (cm >= d) {
                for (; o < stop; o++) {
                    dst[o] = src[o];
                    if (V) vdst[o] = vsrc[o];
                }
            } else {
                const uint32_t m = off[cm];
                const uint32_t l = merge_path(src, s, m, e, o - s);
                serial_merge<K, V>(src, dst, vsrc, vdst, s + l, m, m + (o - s) - l, e, o, stop);
                o = stop;
            }
            c0 = c1;
        }
    }
}

// Round 0 of a unit whose slices sit at their own positions pos[c] (as staged
// by the loads): slices (0,1), (2,3), ... are merged into dst at the unit's
// contiguous offsets off[]; a last slice without a partner is copied.
template <typename K, bool V>
__device__ __forceinline__ void unit_round0(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
                                            uint32_t* __restrict__ vdst, const uint32_t* __restrict__ off,
                                            const uint32_t* __restrict__ pos, uint32_t d) {
    const uint32_t total = off[d];
    const uint32_t ipt = chunk_per_thread<kLvlThreads>(total);
    const uint32_t base = threadIdx.x * ipt;
    if (base >= total) return;
    uint32_t o = base;
    const uint32_t oe = min(base + ipt, total);
    uint32_t c0 = 0;
    for (uint32_t c = 2; c < d; c += 2)
        if (off[c] <= o) c0 = c;
    while (o < oe) {
        const uint32_t c1 = min(c0 + 2, d);
        const uint32_t s = off[c0], e = off[c1];
        const uint32_t stop = min(e, oe);
        if (c0 + 1 >= d) {
            const uint32_t p = pos[c0] - s;
            for (; o < stop; o++) {
                dst[o] = src[p + o];
                if (V) vdst[o] = vsrc[p + o];
            }
        } else {
            const uint32_t pa = pos[c0], pb = pos[c0 + 1];
            const uint32_t na = off[c0 + 1] - s, nb = e - off[c0 + 1];
            const uint32_t diag = o - s;
            const uint32_t l = merge_path2(src + pa, na, src + pb, nb, diag);
            serial_merge2<K, V>(src + pa, na, src + pb, nb, V ? vsrc + pa : nullptr, V ? vsrc + pb : nullptr, dst, vdst, l,
                                diag - l, o, stop);
            o = stop;
        }
        c0 = c1;
    }
}

// Level merge: persistent blocks, each over a contiguous range of work units.
// Per unit: read its descriptor (the next one is prefetched), stage its slices
// in shared memory (TMA bulk copies on an mbarrier for the aligned middles),
// merge them in tournament rounds, and store the result with 16-byte stores.
// Three blocks of 256 threads share an SM (two buffers of C + slack elements
// each), so one block's staging overlaps the others' merging.
template <typename K, bool V>
__global__ void __launch_bounds__(kLvlThreads)
    k_level_merge(const UnitDesc* __restrict__ udesc, const uint64_t* __restrict__ ctr, const K* __restrict__ leaf,
                  const uint32_t* __restrict__ vleaf, K* __restrict__ buf0, K* __restrict__ buf1, uint32_t* __restrict__ vbuf0,
                  uint32_t* __restrict__ vbuf1, uint32_t C, uint64_t n, uint32_t* __restrict__ status) {
    extern __shared__ uint4 smem_raw[];
    // two buffers of C elements plus slack: slices are staged with gaps that
    // put each one on the 16-byte grid of its source, and the last round's
    // output is shifted onto the 16-byte grid of its destination
    const uint32_t CP = C + kLvlPad;
    K* La = reinterpret_cast<K*>(smem_raw);
    K* Lb = La + CP;
    uint32_t* vLa = V ? reinterpret_cast<uint32_t*>(Lb + CP) : nullptr;
    uint32_t* vLb = V ? vLa + CP : nullptr;
    __shared__ UnitDesc ring[2];
    __shared__ uint32_t s_pos[kMaxFanIn];
    __shared__ __align__(8) uint64_t s_bar;
    uint32_t phase = 0;
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);

    const uint32_t total_units = (uint32_t)ctr[kCtrUnits];
    const uint32_t per = (total_units + gridDim.x - 1) / gridDim.x;
    const uint32_t u0 = blockIdx.x * per;
    const uint32_t u1 = min(total_units, u0 + per);
    if (u0 < u1 && threadIdx.x < kUnitDescVec)
        reinterpret_cast<uint4*>(&ring[0])[threadIdx.x] = reinterpret_cast<const uint4*>(udesc + u0)[threadIdx.x];
    for (uint32_t u = u0; u < u1; u++) {
        const UnitDesc& D = ring[(u - u0) & 1];
        // the next unit's descriptor is read while this unit is merged
        uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
        if (u + 1 < u1 && threadIdx.x < kUnitDescVec) nxt = reinterpret_cast<const uint4*>(udesc + u + 1)[threadIdx.x];
        __syncthreads();
        const uint32_t total = D.total, d = D.d & 0xFFu;
        if (total > C) {
            if (threadIdx.x == 0) dev_fail(status, kDevRange);
            return;
        }
        bool bad = d > (uint32_t)kMaxFanIn || (uint64_t)D.out_base + total > n;
        for (uint32_t c = 0; c < d && !bad; c++) {
            const uint32_t m0 = D.off[c + 1] - D.off[c];
            const bool rv = (D.flags >> (16 + c)) & 1u;
            bad = m0 > total || (rv ? (m0 > 0 && (D.src[c] >= n || D.src[c] + 1 < m0))
                                    : (uint64_t)D.src[c] + m0 > n);
        }
        if (bad) {
            if (threadIdx.x == 0) dev_fail(status, kDevUnitRange);
            __syncthreads();
            continue;
        }
        const bool odd = D.d >> 31;
        const K* inner = odd ? buf0 : buf1;                 // children sit at depth + 1
        const uint32_t* vinner = odd ? vbuf0 : vbuf1;
        constexpr uint32_t VK = 16 / sizeof(K);
        // ---- stage the slices: slice c lands at s_pos[c], with its element i at
        // the same offset within 16 bytes as in its source, so that the aligned
        // middle of a forward slice is one bulk copy; reversed slices and the
        // unaligned ends are copied element by element (cp.async)
        if (threadIdx.x == 0) {
            uint32_t P = 0, tx = 0;
            for (uint32_t c = 0; c < d; c++) {
                const uint32_t m = D.off[c + 1] - D.off[c];
                const bool lf = (D.flags >> c) & 1u, rv = (D.flags >> (16 + c)) & 1u;
                const K* src = (lf ? leaf : inner) + D.src[c];
                const uint32_t lead = rv ? 0u : (uint32_t)((reinterpret_cast<uintptr_t>(src) & 15u) / sizeof(K));
                s_pos[c] = P + lead;
                if (!rv) {
                    const uint32_t ib = min(m, (VK - lead) & (VK - 1u));
                    tx += (m - ib) / VK * 16u;
                }
                P = (P + lead + m + VK - 1) / VK * VK;
            }
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar, tx);
            for (uint32_t c = 0; c < d; c++) {
                const uint32_t m = D.off[c + 1] - D.off[c];
                const bool lf = (D.flags >> c) & 1u, rv = (D.flags >> (16 + c)) & 1u;
                if (rv) continue;
                const K* src = (lf ? leaf : inner) + D.src[c];
                const uint32_t lead = s_pos[c] % VK;
                const uint32_t ib = min(m, (VK - lead) & (VK - 1u));
                const uint32_t bytes = (m - ib) / VK * 16u;
                if (bytes) bulk_copy_g2s(La + s_pos[c] + ib, src + ib, bytes, &s_bar);
            }
        }
        __syncthreads();
        for (uint32_t c = 0; c < d; c++) {
            const uint32_t m = D.off[c + 1] - D.off[c], s0 = D.src[c], pc = s_pos[c];
            const bool lf = (D.flags >> c) & 1u, rv = (D.flags >> (16 + c)) & 1u;
            const K* srck = lf ? leaf : inner;
            const uint32_t* srcv = lf ? vleaf : vinner;
            if (rv) {
                for (uint32_t i = threadIdx.x; i < m; i += kLvlThreads) {
                    cp_async<sizeof(K)>(La + pc + i, srck + (s0 - i));
                    if (V) cp_async<4>(vLa + pc + i, srcv + (s0 - i));
                }
            } else {
                const uint32_t lead = pc % VK;
                const uint32_t ib = min(m, (VK - lead) & (VK - 1u));
                const uint32_t ie = ib + (m - ib) / VK * VK;
                for (uint32_t i = threadIdx.x; i < ib; i += kLvlThreads) cp_async<sizeof(K)>(La + pc + i, srck + s0 + i);
                for (uint32_t i = ie + threadIdx.x; i < m; i += kLvlThreads) cp_async<sizeof(K)>(La + pc + i, srck + s0 + i);
                if (V)
                    for (uint32_t i = threadIdx.x; i < m; i += kLvlThreads) cp_async<4>(vLa + pc + i, srcv + s0 + i);
            }
        }
        cp_async_commit();
        cp_async_wait<0>();
        {
            uint32_t spins = 0;
            bool done = mbar_try_wait(&s_bar, phase);
            while (!done && spins < kMbarSpinLimit) {
                done = mbar_try_wait(&s_bar, phase);
                spins++;
            }
            if (__syncthreads_or(!done)) {
                // The bulk copies did not complete: report it, give them one more
                // bounded wait, and stop (the whole block leaves together).  Every copy
                // is well formed by construction (16-byte aligned ends, sizes that are
                // multiples of 16 inside the unit's buffer, the expected byte count set
                // before they are issued), so they complete unless the memory system
                // fails; this branch only keeps that case from hanging the GPU.
                if (threadIdx.x == 0) dev_fail(status, kDevSpin);
                for (spins = 0; !mbar_try_wait(&s_bar, phase) && spins < kMbarSpinLimit; spins++) {
                }
                return;
            }
            phase ^= 1u;
        }
        K* out = odd ? buf1 : buf0;
        uint32_t* vout = odd ? vbuf1 : vbuf0;
        const uint32_t ob = D.out_base;
        // the last round writes element q at shift + q, where shift puts it on
        // the 16-byte grid of out[ob + q] (16-byte stores below)
        const uint32_t shk = (uint32_t)((reinterpret_cast<uintptr_t>(out + ob) & 15u) / sizeof(K));
        const uint32_t shv = V ? (uint32_t)((reinterpret_cast<uintptr_t>(vout + ob) & 15u) / 4u) : 0u;
        uint32_t nr = 0;
        while ((1u << nr) < d) nr++;
        K* cur = La;
        K* oth = Lb;
        uint32_t* vcur = vLa;
        uint32_t* voth = vLb;
        for (uint32_t t = 0; t < nr; t++) {
            const bool last = t + 1 == nr;
            K* dk = oth + (last ? shk : 0u);
            uint32_t* dv = V ? voth + (last ? shv : 0u) : nullptr;
            if (t == 0) unit_round0<K, V>(cur, dk, vcur, dv, D.off, s_pos, d);
            else unit_round<K, V>(cur, dk, vcur, dv, D.off, d, t);
            __syncthreads();
            oth = cur; cur = dk;
            voth = vcur; vcur = dv;
        }
        if (nr) {
            store_vec<K>(out + ob, cur, total, shk);
            if (V) store_vec<uint32_t>(vout + ob, vcur, total, shv);
        } else {
            for (uint32_t q = threadIdx.x; q < total; q += kLvlThreads) {
                out[ob + q] = cur[q];
                if (V) vout[ob + q] = vcur[q];
            }
        }
        if (u + 1 < u1 && threadIdx.x < kUnitDescVec) reinterpret_cast<uint4*>(&ring[(u + 1 - u0) & 1])[threadIdx.x] = nxt;
        __syncthreads();
    }
}

// An input that is a single run (r = 1, read on the device) is the sorted
// output itself, reversed if strictly descending; any other input leaves at once.
template <typename K, bool V>
__global__ void k_copy_single_run(const K* __restrict__ in, const uint32_t* __restrict__ vin, K* __restrict__ out,
                                  uint32_t* __restrict__ vout, uint64_t n, const uint8_t* __restrict__ rdesc,
                                  const uint64_t* __restrict__ ctr) {
    if (ctr[kCtrR] != 1) return;
    const bool rev = rdesc[0] != 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = rev ? n - 1 - i : i;
        out[i] = in[s];
        if (V) vout[i] = vin[s];
    }
}

// Batch: run i is alone in its array iff both of its boundaries carry power 0
// (array starts, or the virtual boundaries 0 and r).  One warp per such run.
template <typename K, bool V>
__global__ void k_copy_lone_runs(const K* __restrict__ in, const uint32_t* __restrict__ vin, K* __restrict__ out,
                                 uint32_t* __restrict__ vout, const uint32_t* __restrict__ rs, const uint8_t* __restrict__ rdesc,
                                 const uint8_t* __restrict__ P, const uint64_t* __restrict__ ctr, uint64_t n) {
    const uint32_t r = (uint32_t)ctr[kCtrR];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < r; i += nwarps) {
        if (P[i] != 0 || P[i + 1] != 0) continue;
        const uint32_t a = rs[i], len = rs[i + 1] - a;
        if ((uint64_t)a + len > n) {
            if (lane == 0) dev_fail(const_cast<uint32_t*>(reinterpret_cast<const uint32_t*>(ctr + kCtrStatus)), kDevLoneRange);
            continue;
        }
        const bool rev = rdesc[i] != 0;
        for (uint32_t q = lane; q < len; q += 32) {
            const uint32_t src = rev ? a + len - 1 - q : a + q;
            out[a + q] = in[src];
            if (V) vout[a + q] = vin[src];
        }
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

MergeGeom merge_geom(int key_bytes, bool vals, int k, int tile) {
    // {fused tile, level unit} elements per choice
    static const uint32_t kKeys4[kTileChoices][2] = {{4096, 9216}, {6144, 9216}, {2048, 4096}};
    static const uint32_t kMid[kTileChoices][2] = {{4096, 4096}, {2048, 3072}, {1536, 2048}};
    static const uint32_t kKeys8Vals[kTileChoices][2] = {{3072, 4096}, {2048, 3072}, {1024, 2048}};
    const uint32_t(*t)[2] = (key_bytes == 4 && !vals) ? kKeys4 : ((key_bytes == 8 && vals) ? kKeys8Vals : kMid);
    const int c = tile < 0 || tile >= kTileChoices ? 0 : tile;
    MergeGeom g;
    g.c_fused = t[c][0];
    g.c_level = t[c][1];
    g.tmax = g.c_fused;
    g.ts = g.c_level / (uint32_t)k;
    g.k = k;
    // persistent level merge: two buffers of c_level elements per block
    size_t lvl_smem = (size_t)2 * (g.c_level + kLvlPad) * ((size_t)key_bytes + (vals ? 4 : 0)) + 256;
    g.level_grid = 152 * (uint32_t)std::min<size_t>(16, (220 * 1024) / lvl_smem);
    size_t fz_smem = (size_t)2 * (g.c_fused + kFusedPad) * ((size_t)key_bytes + (vals ? 4 : 0)) +
                     (size_t)2 * (g.c_fused / 2 + 8) * 4 + 1024;
    g.fused_grid = 152 * (uint32_t)std::max<size_t>(1, std::min<size_t>(8, (220 * 1024) / fz_smem));
    return g;
}

template <typename K, bool V>
void launch_fused(const K* leaf_keys, const uint32_t* leaf_vals, K* out, uint32_t* vout, uint64_t nfused,
                  const MergeGeom& g, const WsView& ws, cudaStream_t st) {
    size_t smem = FusedSmem<K, V>::bytes(g.c_fused);
    cudaFuncSetAttribute(k_fused<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint32_t grid = (uint32_t)std::min<uint64_t>(nfused, g.fused_grid);
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    k_fused<K, V><<<grid, kFusedThreads, smem, st>>>(ws.fused_list, ws.counters, leaf_keys, leaf_vals, out, tmp, vout,
                                                     ws.vals_tmp, ws.run_starts, ws.run_desc, ws.powers, g.c_fused, g.k,
                                                     ws.n, reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus),
                                                     reinterpret_cast<unsigned long long*>(ws.counters + kCtrFusedNext));
    g_launches += 1;
}

template <typename K>
void launch_level_plan(int p, uint32_t nn_bound, uint64_t elems_bound, int k, const K* leaf_keys, K* out,
                       const MergeGeom& g, const WsView& ws, cudaStream_t st) {
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    k_level_count<<<(uint32_t)std::min<uint64_t>(ceil_div(std::max<uint32_t>(nn_bound, 1), 256), 152 * 4), 256, 0, st>>>(
        ws.nodes_lvl, ws.level_off, p, ws.run_starts, g.ts, ws.counters);
    k_level_prep<<<1, 1024, 0, st>>>(ws.nodes_lvl, ws.level_off, p, ws.counters, ws.unit_node);
    const uint64_t split_bound = elems_bound / g.ts + 1;
    const uint32_t split_blocks = (uint32_t)std::min<uint64_t>(ceil_div(split_bound * (uint64_t)k, 256), 152 * 16);
    k_level_split<K><<<split_blocks, 256, 0, st>>>(ws.nodes_lvl, ws.level_off, p, ws.counters, ws.run_starts, ws.run_desc,
                                                    leaf_keys, out, tmp, g.ts, k, ws.unit_node, ws.split_tab);
    const uint64_t ivl_bound = split_bound + nn_bound;
    const uint32_t tiles = (uint32_t)ceil_div(ivl_bound, kPackTile);
    k_interval_size<<<(uint32_t)std::min<uint64_t>(ceil_div(ivl_bound, 256), 152 * 8), 256, 0, st>>>(
        ws.nodes_lvl, ws.level_off, p, ws.unit_node, ws.split_tab, ws.counters, k, ws.ivl_size);
    k_pack_reduce<<<tiles, kPackThreads, 0, st>>>(ws.ivl_size, ws.counters, g.c_level, ws.pack_tiles);
    k_pack_scan<<<1, 1024, 0, st>>>(ws.pack_tiles, tiles, ws.counters);
    k_pack_apply<<<tiles, kPackThreads, 0, st>>>(ws.ivl_size, ws.counters, g.c_level, ws.pack_tiles, ws.unit_first);
    const uint32_t desc_blocks = (uint32_t)std::min<uint64_t>(ceil_div(ivl_bound, 256), 152 * 16);
    k_level_desc<<<desc_blocks, 256, 0, st>>>(ws.nodes_lvl, ws.level_off, p, ws.unit_node, ws.unit_first, ws.split_tab,
                                              ws.counters, ws.run_starts, ws.run_desc, k,
                                              reinterpret_cast<UnitDesc*>(ws.unit_desc));
    g_launches += 8;
}

template <typename K, bool V>
void launch_level_merge(uint32_t nn_bound, uint64_t elems_bound, const K* leaf_keys, const uint32_t* leaf_vals, K* out,
                        uint32_t* vout, const MergeGeom& g, const WsView& ws, cudaStream_t st) {
    K* tmp = reinterpret_cast<K*>(ws.keys_tmp);
    const uint64_t bound = elems_bound / g.ts + nn_bound + 1;
    size_t smem = (size_t)2 * (g.c_level + kLvlPad) * (sizeof(K) + (V ? 4 : 0));
    cudaFuncSetAttribute(k_level_merge<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    uint32_t grid = (uint32_t)std::min<uint64_t>(bound, (uint64_t)g.level_grid);
    k_level_merge<K, V><<<grid, kLvlThreads, smem, st>>>(reinterpret_cast<const UnitDesc*>(ws.unit_desc), ws.counters,
                                                          leaf_keys, leaf_vals, out, tmp, vout, ws.vals_tmp, g.c_level,
                                                          ws.n, reinterpret_cast<uint32_t*>(ws.counters + kCtrStatus));
    g_launches += 1;
}

template <typename K, bool V>
void launch_copy_single_run(const K* in, const uint32_t* vin, K* out, uint32_t* vout, uint64_t n, const WsView& ws,
                            cudaStream_t st) {
    uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(n, 256), 152 * 8);
    k_copy_single_run<K, V><<<grid, 256, 0, st>>>(in, vin, out, vout, n, ws.run_desc, ws.counters);
    g_launches += 1;
}

template <typename K, bool V>
void launch_copy_lone_runs(const K* in, const uint32_t* vin, K* out, uint32_t* vout, uint32_t r_bound, const WsView& ws,
                           cudaStream_t st) {
    uint32_t blocks = (uint32_t)std::min<uint64_t>(ceil_div((uint64_t)r_bound * 32, 256), 152 * 8);
    k_copy_lone_runs<K, V><<<blocks, 256, 0, st>>>(in, vin, out, vout, ws.run_starts, ws.run_desc, ws.powers, ws.counters,
                                                    ws.n);
    g_launches += 1;
}

#define MPS_INST(K, V)                                                                                                  \
    template void launch_fused<K, V>(const K*, const uint32_t*, K*, uint32_t*, uint64_t, const MergeGeom&,             \
                                     const WsView&, cudaStream_t);                                                      \
    template void launch_level_merge<K, V>(uint32_t, uint64_t, const K*, const uint32_t*, K*, uint32_t*,               \
                                           const MergeGeom&, const WsView&, cudaStream_t);                              \
    template void launch_copy_single_run<K, V>(const K*, const uint32_t*, K*, uint32_t*, uint64_t, const WsView&,      \
                                               cudaStream_t);                                                           \
    template void launch_copy_lone_runs<K, V>(const K*, const uint32_t*, K*, uint32_t*, uint32_t, const WsView&,       \
                                              cudaStream_t);
MPS_INST(uint32_t, false)
MPS_INST(uint32_t, true)
MPS_INST(uint64_t, false)
MPS_INST(uint64_t, true)
#undef MPS_INST
template void launch_level_plan<uint32_t>(int, uint32_t, uint64_t, int, const uint32_t*, uint32_t*, const MergeGeom&,
                                          const WsView&, cudaStream_t);
template void launch_level_plan<uint64_t>(int, uint32_t, uint64_t, int, const uint64_t*, uint64_t*, const MergeGeom&,
                                          const WsView&, cudaStream_t);

}  // namespace mps
