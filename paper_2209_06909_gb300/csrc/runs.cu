// runs.cu -- run detection (Sec. 2) and boundary powers (Def. 3.1).
//
// Run detection.  The paper finds runs with a greedy left-to-right scan
// (FirstRunOf in Alg. 2): a run is the maximal strictly decreasing prefix if
// its first two elements decrease, otherwise the maximal weakly increasing
// prefix.  Whether element i starts a run depends on the direction of the run
// in progress, so the scan is written as a 3-state automaton
//     B = element starts a run, A = inside an ascending run, D = inside a
//     strictly descending run,
// driven by lt_i = (key[i] < key[i-1]):
//     not lt : B->A, A->A, D->B          lt : B->D, A->B, D->D
// and element 0 is always B.  A tile's effect is a map {B,A,D} -> {B,A,D}
// plus, per entry state, the number of B states produced; maps compose
// associatively, so the greedy scan becomes a scan over tiles: each tile
// summarises its elements, one block composes the summaries into every tile's
// entry state and run offset, and each tile then writes its runs.  Run i is
// descending iff key[s_i + 1] < key[s_i].
//
// Powers.  With run i-1 = [s_{i-1}, s_i) and run i = [s_i, s_{i+1}), Def. 3.1's
// midpoints are a = (s_{i-1} + s_i) / 2n and b = (s_i + s_{i+1}) / 2n.  For a
// w with 2^w >= n put x = floor(a 2^w), y = floor(b 2^w) (exact integer
// quotients).  Because floor(floor(z)/m) = floor(z/m), floor(a 2^q) = x >> (w-q)
// for q <= w, so the 2-way power -- the least q with floor(a 2^q) < floor(b 2^q)
// -- is w minus the index of the highest bit where x and y differ; b - a >= 1/n
// guarantees x != y.  The predicate is monotone in q, so for k = 2^t the k-way
// power is ceil(P2 / t) (the "squish" of Sec. 3.1 for t = 2).
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mps {

namespace {

constexpr int kDetThreads = 256;
constexpr int kDetItems = 32;
static_assert(kDetThreads * kDetItems == kDetTile, "detection tile");

// Smallest array start >= x among off[0..m] (a batch of m arrays laid end to
// end), or ~0 if none.  Without a batch (off == nullptr) element 0 is the only
// start.
__device__ __forceinline__ uint64_t next_start(const uint64_t* __restrict__ off, uint32_t m, uint64_t x) {
    if (off == nullptr) return x == 0 ? 0ull : ~0ull;
    uint32_t lo = 0, hi = m + 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (off[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo <= m ? off[lo] : ~0ull;
}

__device__ __forceinline__ uint32_t step_state(uint32_t s, bool lt) {
    // B = 0, A = 1, D = 2
    return lt ? (s == 1u ? 0u : 2u) : (s == 2u ? 0u : 1u);
}

// Summary of a segment: map (2 bits per entry state) and B-counts per entry state.
struct RunSum { uint32_t map, c0, c1, c2; };

__device__ __forceinline__ uint32_t map_get(uint32_t m, uint32_t q) { return (m >> (2 * q)) & 3u; }

struct OpRunSum {
    __device__ uint4 operator()(uint4 X, uint4 Y) const {
        uint4 o;
        uint32_t cy[3] = {Y.y, Y.z, Y.w};
        uint32_t m0 = map_get(X.x, 0), m1 = map_get(X.x, 1), m2 = map_get(X.x, 2);
        o.x = map_get(Y.x, m0) | (map_get(Y.x, m1) << 2) | (map_get(Y.x, m2) << 4);
        o.y = X.y + cy[m0];
        o.z = X.z + cy[m1];
        o.w = X.w + cy[m2];
        return o;
    }
};

__device__ __forceinline__ uint4 runsum_identity() { return make_uint4(0u | (1u << 2) | (2u << 4), 0u, 0u, 0u); }

// Loads keys[i0-1 .. i0+kDetItems] (kDetItems + 2 values) with bounds checks.
template <typename K>
__device__ __forceinline__ void load_window(const K* __restrict__ keys, uint64_t n, uint64_t i0, K (&v)[kDetItems + 2]) {
    v[0] = (i0 >= 1 && i0 - 1 < n) ? keys[i0 - 1] : K(0);
    if (i0 + kDetItems <= n && (reinterpret_cast<uintptr_t>(keys + i0) & 15u) == 0) {
        constexpr int kVec = 16 / sizeof(K);
        const uint4* p = reinterpret_cast<const uint4*>(keys + i0);
#pragma unroll
        for (int q = 0; q < kDetItems / kVec; q++) {
            uint4 w = __ldg(p + q);
            const K* e = reinterpret_cast<const K*>(&w);
#pragma unroll
            for (int t = 0; t < kVec; t++) v[1 + q * kVec + t] = e[t];
        }
    } else {
#pragma unroll
        for (int j = 0; j < kDetItems; j++) v[1 + j] = (i0 + j < n) ? keys[i0 + j] : K(0);
    }
    v[kDetItems + 1] = (i0 + kDetItems < n) ? keys[i0 + kDetItems] : K(0);
}

// Bit j (j = 0..32) = key[i0 + j] < key[i0 + j - 1]: the comparisons that
// drive the automaton for the thread's 32 elements, plus one more for the
// direction of a run that starts at its last element.
template <typename K>
__device__ __forceinline__ uint64_t lt_mask(const K (&v)[kDetItems + 2]) {
    uint64_t msk = 0;
#pragma unroll
    for (int j = 0; j <= kDetItems; j++) msk |= (uint64_t)(v[1 + j] < v[j] ? 1u : 0u) << j;
    return msk;
}

// A thread's 32 elements under the automaton, for each entry state s in
// {B, A, D}: the start masks ms[s] (bit j: element i0 + j starts a run), and
// the summary (exit-state map, starts per entry state).  Also the directions:
// bit j of *dm = a run starting at element i0 + j is strictly decreasing.
// Without an array start inside the chunk, each 8-element quarter is one
// lookup in lut[state * 256 + comparison bits] = start mask | exit state << 8;
// otherwise (batches) the automaton steps element by element.
struct ThreadRuns {
    uint4 sum;
    uint32_t ms[3];
    uint32_t dm;
};

__device__ __forceinline__ ThreadRuns thread_runs(uint64_t lt, uint64_t n, uint64_t i0, const uint64_t* __restrict__ off,
                                                  uint32_t m, const uint16_t* __restrict__ lut) {
    ThreadRuns R;
    uint64_t nx = next_start(off, m, i0);
    if (i0 + kDetItems <= n && nx >= i0 + kDetItems && i0 != nx) {
        uint32_t map = 0;
#pragma unroll
        for (uint32_t st = 0; st < 3; st++) {
            uint32_t s = st, msk = 0;
#pragma unroll
            for (int q = 0; q < kDetItems / 8; q++) {
                const uint32_t e = lut[s * 256 + (uint32_t)((lt >> (8 * q)) & 0xFFu)];
                msk |= (e & 0xFFu) << (8 * q);
                s = e >> 8;
            }
            R.ms[st] = msk;
            map |= s << (2 * st);
        }
        R.sum = make_uint4(map, __popc(R.ms[0]), __popc(R.ms[1]), __popc(R.ms[2]));
        // the element after the chunk must exist and be in the same array
        const bool tail_ok = i0 + kDetItems < n && nx != i0 + kDetItems;
        R.dm = (uint32_t)(lt >> 1) & (tail_ok ? 0xFFFFFFFFu : 0x7FFFFFFFu);
        return R;
    }
    uint32_t s0 = 0, s1 = 1, s2 = 2, m0 = 0, m1 = 0, m2 = 0, dm = 0;
#pragma unroll
    for (int j = 0; j < kDetItems; j++) {
        const uint64_t i = i0 + j;
        if (i < n) {
            if (i == nx) {
                nx = next_start(off, m, i + 1);
                s0 = s1 = s2 = 0;
            } else {
                const bool l = (lt >> j) & 1u;
                s0 = step_state(s0, l); s1 = step_state(s1, l); s2 = step_state(s2, l);
            }
            m0 |= (s0 == 0 ? 1u : 0u) << j;
            m1 |= (s1 == 0 ? 1u : 0u) << j;
            m2 |= (s2 == 0 ? 1u : 0u) << j;
            // descending iff the next element is in the same array and smaller
            if (i + 1 < n && i + 1 != nx && ((lt >> (j + 1)) & 1u)) dm |= 1u << j;
        }
    }
    R.ms[0] = m0; R.ms[1] = m1; R.ms[2] = m2;
    R.dm = dm;
    R.sum = make_uint4(s0 | (s1 << 2) | (s2 << 4), __popc(m0), __popc(m1), __popc(m2));
    return R;
}

__device__ __forceinline__ uint32_t runsum_count(uint4 a, uint32_t st) { return st == 0 ? a.y : (st == 1 ? a.z : a.w); }

// ---- run detection in three passes over tiles of kDetTile elements
// 1. every tile: the comparison bits of its elements (one 32-bit word per
//    thread, bit j = key[i0+j] < key[i0+j-1]) and the tile's summary (exit
//    state per entry state, starts per entry state);
// 2. one block: the exclusive composition of the tile summaries, i.e. each
//    tile's entry state and first run index (element 0 enters in state B);
// 3. every tile: the run starts and directions from its comparison bits and
//    entry state, staged in shared memory and written as one coalesced range.
// The keys are read once; passes 2 and 3 read n/8 bytes of comparison bits.

// lut[state * 256 + comparison bits of 8 elements] = start mask | exit state << 8,
// generated at compile time and copied to shared memory by every block.
struct DetLut {
    uint16_t v[3 * 256];
};
constexpr DetLut make_det_lut() {
    DetLut t{};
    for (uint32_t e = 0; e < 3 * 256; e++) {
        uint32_t st = e >> 8, msk = 0;
        for (uint32_t j = 0; j < 8; j++) {
            const bool lt = ((e >> j) & 1u) != 0;
            st = lt ? (st == 1u ? 0u : 2u) : (st == 2u ? 0u : 1u);  // the automaton above
            msk |= (st == 0 ? 1u : 0u) << j;
        }
        t.v[e] = (uint16_t)(msk | (st << 8));
    }
    return t;
}
__device__ const DetLut kDetLut = make_det_lut();
static_assert(sizeof(DetLut) == 3 * 256 * 2 && sizeof(DetLut) % 16 == 0, "16-byte copies of the table");

__device__ __forceinline__ void build_lut(uint16_t* lut) {
    const uint4* src = reinterpret_cast<const uint4*>(kDetLut.v);
    for (uint32_t q = threadIdx.x; q < sizeof(DetLut) / 16; q += blockDim.x) reinterpret_cast<uint4*>(lut)[q] = src[q];
}

// One block per tile.
template <typename K>
__global__ void __launch_bounds__(kDetThreads) k_detect_sum(const K* __restrict__ keys, uint64_t n,
                                                            const uint64_t* __restrict__ off, uint32_t m,
                                                            uint32_t* __restrict__ lt_words, uint4* __restrict__ tile_sum) {
    __shared__ uint4 tmp[kDetThreads / 32 + 1];
    __shared__ __align__(16) uint16_t s_lut[3 * 256];
    const uint32_t tile = blockIdx.x;
    const uint64_t i0 = (uint64_t)tile * kDetTile + (uint64_t)threadIdx.x * kDetItems;
    uint64_t lt;
    {
        // the keys are requested first; the table copy overlaps their latency
        K v[kDetItems + 2];
        load_window(keys, n, i0, v);
        build_lut(s_lut);
        lt = lt_mask(v);
    }
    if (i0 < n) lt_words[(size_t)tile * kDetThreads + threadIdx.x] = (uint32_t)lt;
    __syncthreads();
    const ThreadRuns tr = thread_runs(lt, n, i0, off, m, s_lut);
    uint4 tot;
    block_scan_excl<kDetThreads, false>(tr.sum, OpRunSum(), runsum_identity(), tmp, &tot);
    if (threadIdx.x == 0) tile_sum[tile] = tot;
}

// One block of 1024 threads over all tiles: tile_pre[t] = (entry state, runs
// before tile t); writes r and the end sentinel run_starts[r] = n.  Warp w
// owns a contiguous range of tiles and walks it 32 tiles at a time (coalesced
// 16-byte loads, an in-warp scan, a carry); one block scan joins the warps.
__device__ __forceinline__ uint4 warp_scan_incl(uint4 x) {
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint4 y = shfl_up(x, o);
        if (lane >= (uint32_t)o) x = OpRunSum()(y, x);
    }
    return x;
}
__device__ __forceinline__ uint4 shfl_idx(uint4 v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src); v.y = __shfl_sync(0xffffffffu, v.y, src);
    v.z = __shfl_sync(0xffffffffu, v.z, src); v.w = __shfl_sync(0xffffffffu, v.w, src);
    return v;
}

__global__ void __launch_bounds__(1024) k_detect_scan(uint64_t n, const uint4* __restrict__ tile_sum, uint2* __restrict__ tile_pre,
                                                      uint64_t* __restrict__ counters, uint32_t* __restrict__ run_starts) {
    __shared__ uint4 s_warp[32];
    __shared__ uint4 tmp[1024 / 32 + 1];
    const uint32_t tiles = (uint32_t)ceil_div(n, kDetTile);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t per = (tiles + 31) / 32;  // tiles per warp
    const uint32_t t0 = min(tiles, warp * per), t1 = min(tiles, t0 + per);
    // pass 1: the warp's aggregate (the next 32 summaries are loaded while
    // the current ones are scanned)
    uint4 carry = runsum_identity();
    uint4 nx = t0 + lane < t1 ? tile_sum[t0 + lane] : runsum_identity();
    for (uint32_t b = t0; b < t1; b += 32) {
        const uint4 cur = nx;
        nx = b + 32 + lane < t1 ? tile_sum[b + 32 + lane] : runsum_identity();
        const uint4 x = warp_scan_incl(cur);
        carry = OpRunSum()(carry, shfl_idx(x, 31));
    }
    uint4 tot;
    const uint4 wpre = block_scan_excl<1024, false>(lane == 0 ? carry : runsum_identity(), OpRunSum(), runsum_identity(), tmp,
                                                    &tot);
    if (lane == 0) s_warp[warp] = wpre;
    __syncthreads();
    // pass 2: every tile's exclusive prefix, entered in state B
    carry = s_warp[warp];
    nx = t0 + lane < t1 ? tile_sum[t0 + lane] : runsum_identity();
    for (uint32_t b = t0; b < t1; b += 32) {
        const uint32_t t = b + lane;
        const uint4 x = nx;
        nx = b + 32 + lane < t1 ? tile_sum[b + 32 + lane] : runsum_identity();
        const uint4 incl = warp_scan_incl(x);
        uint4 excl = shfl_up(incl, 1);
        if (lane == 0) excl = runsum_identity();
        const uint4 pre = OpRunSum()(carry, excl);
        if (t < t1) tile_pre[t] = make_uint2(map_get(pre.x, 0), pre.y);
        carry = OpRunSum()(carry, shfl_idx(incl, 31));
    }
    if (threadIdx.x == 0) {
        counters[kCtrR] = tot.y;
        run_starts[tot.y] = (uint32_t)n;
    }
}

// One block per tile.
__global__ void __launch_bounds__(kDetThreads) k_detect_write(uint64_t n, const uint64_t* __restrict__ off, uint32_t m,
                                                              const uint32_t* __restrict__ lt_words, const uint2* __restrict__ tile_pre,
                                                              uint32_t* __restrict__ run_starts, uint8_t* __restrict__ run_desc) {
    __shared__ uint4 tmp[kDetThreads / 32 + 1];
    __shared__ uint32_t s_rs[kDetTile];
    __shared__ uint8_t s_rd[kDetTile];
    __shared__ __align__(16) uint16_t s_lut[3 * 256];
    build_lut(s_lut);
    const uint32_t tile = blockIdx.x;
    const uint64_t i0 = (uint64_t)tile * kDetTile + (uint64_t)threadIdx.x * kDetItems;
    const uint64_t words = ceil_div(n, kDetItems);
    const uint64_t gi = (uint64_t)tile * kDetThreads + threadIdx.x;
    uint64_t lt = 0;
    if (gi < words) {
        lt = lt_words[gi];
        // bit 32 (the comparison after the chunk) is bit 0 of the next chunk's word
        if (gi + 1 < words) lt |= (uint64_t)(lt_words[gi + 1] & 1u) << 32;
    }
    __syncthreads();
    const ThreadRuns tr = thread_runs(lt, n, i0, off, m, s_lut);
    uint4 tot;
    const uint4 pre = block_scan_excl<kDetThreads, false>(tr.sum, OpRunSum(), runsum_identity(), tmp, &tot);
    const uint2 tp = tile_pre[tile];
    const uint32_t st_in = tp.x, base = tp.y;
    const uint32_t st = map_get(pre.x, st_in);  // state entering this thread's chunk
    uint32_t msk = st == 0 ? tr.ms[0] : (st == 1 ? tr.ms[1] : tr.ms[2]);
    uint32_t idx = runsum_count(pre, st_in);
    while (msk) {
        const uint32_t j = __ffs(msk) - 1;
        msk &= msk - 1;
        s_rs[idx] = (uint32_t)(i0 + j);
        s_rd[idx] = (uint8_t)((tr.dm >> j) & 1u);
        idx++;
    }
    __syncthreads();
    const uint32_t cnt = runsum_count(tot, st_in);
    for (uint32_t q = threadIdx.x; q < cnt; q += kDetThreads) {
        run_starts[base + q] = s_rs[q];
        run_desc[base + q] = s_rd[q];
    }
}

// Powers of boundaries 1..r-1, sentinels powers[0] = powers[r] = 0, padding
// of 255 up to the next multiple of 32, the bit set of powers that occur and
// the longest run.  Each thread takes 16 boundaries: 16-byte loads of run
// starts (the array is padded past r) and one 16-byte store of powers.
template <uint32_t LOG2K, bool BATCH>
__global__ void __launch_bounds__(256) k_powers(const uint32_t* __restrict__ run_starts, uint64_t* __restrict__ counters,
                                                uint64_t n, uint32_t w, uint64_t magic,
                                                const uint64_t* __restrict__ off, uint32_t m,
                                                const uint2* __restrict__ arr_param,
                                                uint8_t* __restrict__ powers, unsigned long long* __restrict__ level_bits) {
    __shared__ unsigned long long red[256 / 32 + 1];
    __shared__ uint32_t redm[256 / 32 + 1];
    const uint32_t r = (uint32_t)counters[kCtrR];
    const uint32_t groups = (r + 1 + 15) / 16;  // boundaries 0..r
    const uint32_t pad_end = (r + 1 + 31) / 32 * 32;
    unsigned long long bits = 0;
    uint32_t longest = 0;  // longest run seen by this thread
    // a single array: n and its shift are the same for every boundary
    const bool pow2_1 = (n & (n - 1)) == 0;
    const int sh1 = (int)w - (int)__ffsll((long long)n);  // w - log2(2n) when n is a power of two
    for (uint32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < groups; gi += gridDim.x * blockDim.x) {
        const uint32_t i0 = gi * 16;
        uint32_t rv[20];
        const uint4* r4 = reinterpret_cast<const uint4*>(run_starts + i0);
#pragma unroll
        for (int q = 0; q < 5; q++) {
            const uint4 x = r4[q];
            rv[4 * q] = x.x; rv[4 * q + 1] = x.y; rv[4 * q + 2] = x.z; rv[4 * q + 3] = x.w;
        }
        const uint32_t prev = i0 ? run_starts[i0 - 1] : 0u;
        // the array holding run i0 (a batch sorts each array on its own): last a with off[a] <= s
        uint32_t arr = 0;
        if (BATCH) {
            uint32_t lo = 0, hi = m + 1;
            const uint32_t s0 = rv[0];
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (off[mid] <= s0) lo = mid; else hi = mid;
            }
            arr = lo;
        }
        uint32_t word[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int q = 0; q < 16; q++) {
            const uint32_t i = i0 + q;
            uint32_t pk = 255u;  // padding past r
            if (i <= r) {
                const uint32_t si = rv[q];
                const uint32_t sp = q ? rv[q - 1] : prev;
                if (i >= 1) longest = max(longest, si - sp);
                pk = 0;
                uint64_t base = 0, nn = n;
                uint32_t ww = w;
                uint64_t mg = magic;
                bool arr_start = false;
                if (BATCH && i >= 1 && i < r) {
                    while (arr < m && off[arr + 1] <= si) arr++;
                    base = off[arr];
                    nn = off[arr + 1] - base;
                    arr_start = (base == si);
                    const uint2 prm = arr_param[arr];
                    ww = prm.x;
                    mg = ((uint64_t)prm.y << 32) | arr_param[m + arr].x;
                }
                if (i >= 1 && i < r && !arr_start) {
                    const uint64_t d = BATCH ? nn : n;
                    const uint64_t a2 = (uint64_t)(sp - base) + (si - base);         // 2n * a  (< 2n < 2^33)
                    const uint64_t b2 = (uint64_t)(si - base) + (rv[q + 1] - base);  // 2n * b
                    uint32_t h;
                    if (BATCH ? (d & (d - 1)) == 0 : pow2_1) {
                        // n a power of two (so n <= 2^31 and a2, b2 < 2^32): x = a2 * 2^w / 2n
                        // is a shift, and x, y < 2^w <= 2^31
                        const int sh = BATCH ? (int)ww - (int)__ffsll((long long)d) : sh1;
                        const uint32_t a32 = (uint32_t)a2, b32 = (uint32_t)b2;
                        const uint32_t x = sh >= 0 ? a32 << sh : a32 >> -sh;
                        const uint32_t y = sh >= 0 ? b32 << sh : b32 >> -sh;
                        h = 31u - (uint32_t)__clz((int)(x ^ y));
                    } else {
                        // x = a2 * 2^(w-1) / n, the same quotient as a2 * 2^w / 2n, with the
                        // product below 2^64 for n < 2^32 (a2 < 2^33, 2^(w-1) <= 2^31);
                        // mg = floor((2^64 - 1) / n) gives it to within two, then corrected
                        const uint64_t X = a2 << (ww - 1), Y = b2 << (ww - 1);
                        uint64_t x = __umul64hi(X, mg), y = __umul64hi(Y, mg);
                        uint64_t rx = X - x * d, ry = Y - y * d;
                        while (rx >= d) { x++; rx -= d; }
                        while (ry >= d) { y++; ry -= d; }
                        h = 63u - (uint32_t)__clzll((long long)(x ^ y));
                    }
                    const uint32_t p2 = ww - h;
                    pk = (p2 + LOG2K - 1) / LOG2K;  // ceil(P_2 / log2 k): the power for fan-in k
                    bits |= 1ull << pk;
                }
            }
            word[q >> 2] |= pk << (8 * (q & 3));
        }
        *reinterpret_cast<uint4*>(powers + i0) = make_uint4(word[0], word[1], word[2], word[3]);
        if (i0 <= r && r < i0 + 16 && pad_end > i0 + 16)
            *reinterpret_cast<uint4*>(powers + i0 + 16) = make_uint4(~0u, ~0u, ~0u, ~0u);
    }
    bits = block_reduce<256>(bits, OpOrU64(), 0ull, red);
    longest = block_reduce<256>(longest, OpMax32(), 0u, redm);
    if (threadIdx.x == 0 && bits) atomicOr(level_bits, bits);
    if (threadIdx.x == 0 && longest) atomicMax(reinterpret_cast<unsigned long long*>(counters + kCtrMaxRun), (unsigned long long)longest);
}

// Per-array power parameters of a batch: w = ceil(log2 n_a) and the 64-bit
// reciprocal floor((2^64 - 1) / n_a), stored as prm[a] = (w, magic_hi),
// prm[m + a].x = magic_lo.  Also the longest array, checked against the
// caller's bound max_len (0: no bound given).
__global__ void k_array_params(const uint64_t* __restrict__ off, uint32_t m, uint64_t max_len, uint2* __restrict__ prm,
                               uint64_t* __restrict__ counters) {
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) {
        const uint64_t na = off[a + 1] - off[a];
        if (max_len && na > max_len) dev_fail(reinterpret_cast<uint32_t*>(counters + kCtrStatus), kDevMaxLen);
        atomicMax(reinterpret_cast<unsigned long long*>(counters + kCtrMaxLen), (unsigned long long)na);
        uint32_t w = 0;
        while ((1ull << w) < na) w++;
        const uint64_t mg = na ? ~0ull / na : 0ull;
        prm[a] = make_uint2(w, (uint32_t)(mg >> 32));
        prm[m + a] = make_uint2((uint32_t)mg, 0u);
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

template <typename K>
void launch_detect(const K* keys, uint64_t n, const WsView& ws, cudaStream_t st) {
    const uint32_t tiles = (uint32_t)ceil_div(n, kDetTile);
    if (tiles == 0) return;
    // detection scratch: tile summaries (16 B), tile prefixes (8 B), comparison words (4 B per 32 keys)
    uint4* tile_sum = reinterpret_cast<uint4*>(ws.det_state);
    uint2* tile_pre = reinterpret_cast<uint2*>(tile_sum + tiles);
    uint32_t* lt_words = reinterpret_cast<uint32_t*>(tile_pre + tiles);
    k_detect_sum<K><<<tiles, kDetThreads, 0, st>>>(keys, n, ws.batch_off, ws.batch_m, lt_words, tile_sum);
    k_detect_scan<<<1, 1024, 0, st>>>(n, tile_sum, tile_pre, ws.counters, ws.run_starts);
    k_detect_write<<<tiles, kDetThreads, 0, st>>>(n, ws.batch_off, ws.batch_m, lt_words, tile_pre, ws.run_starts, ws.run_desc);
    g_launches += 3;
}

template void launch_detect<uint32_t>(const uint32_t*, uint64_t, const WsView&, cudaStream_t);
template void launch_detect<uint64_t>(const uint64_t*, uint64_t, const WsView&, cudaStream_t);

void launch_powers(uint64_t n, uint32_t r, int k, const WsView& ws, cudaStream_t st) {
    uint32_t w = 0;
    while ((1ull << w) < n) w++;
    uint64_t magic = ~0ull / std::max<uint64_t>(n, 1);
    const uint32_t log2k = (uint32_t)__builtin_ctz((unsigned)k);
    uint32_t threads = 256;
    uint32_t blocks = (uint32_t)std::min<uint64_t>(ceil_div(ceil_div((uint64_t)r + 1, 16), threads), 152 * 16);
    if (ws.batch_off) {
        k_array_params<<<(uint32_t)std::min<uint64_t>(ceil_div(ws.batch_m, 256), 1024), 256, 0, st>>>(ws.batch_off, ws.batch_m,
                                                                                                  ws.batch_max_len, ws.batch_prm,
                                                                                                  ws.counters);
        g_launches += 1;
    }
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(ws.counters + kCtrLevelBits);
#define MPS_POWERS(L2, B)                                                                                             \
    k_powers<L2, B><<<blocks, threads, 0, st>>>(ws.run_starts, ws.counters, n, w, magic, ws.batch_off, ws.batch_m,  \
                                                ws.batch_prm, ws.powers, bits)
    if (ws.batch_off) {
        if (log2k == 1) MPS_POWERS(1, true); else if (log2k == 2) MPS_POWERS(2, true); else if (log2k == 3) MPS_POWERS(3, true); else MPS_POWERS(4, true);
    } else {
        if (log2k == 1) MPS_POWERS(1, false); else if (log2k == 2) MPS_POWERS(2, false); else if (log2k == 3) MPS_POWERS(3, false); else MPS_POWERS(4, false);
    }
#undef MPS_POWERS
    g_launches += 1;
}

}  // namespace mps
