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
// associatively, so the greedy scan becomes a reduce / scan / apply over
// tiles.  Run i is descending iff key[s_i + 1] < key[s_i].
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
constexpr int kDetItems = 16;
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

template <typename K>
__device__ __forceinline__ uint4 thread_runsum(const K (&v)[kDetItems + 2], uint64_t n, uint64_t i0,
                                              const uint64_t* __restrict__ off, uint32_t m) {
    uint32_t s0 = 0, s1 = 1, s2 = 2, c0 = 0, c1 = 0, c2 = 0;
    uint64_t nx = next_start(off, m, i0);
#pragma unroll
    for (int j = 0; j < kDetItems; j++) {
        uint64_t i = i0 + j;
        if (i < n) {
            if (i == nx) {
                nx = next_start(off, m, i + 1);
                s0 = s1 = s2 = 0;
            } else {
                bool lt = v[1 + j] < v[j];
                s0 = step_state(s0, lt); s1 = step_state(s1, lt); s2 = step_state(s2, lt);
            }
            c0 += (s0 == 0); c1 += (s1 == 0); c2 += (s2 == 0);
        }
    }
    return make_uint4(s0 | (s1 << 2) | (s2 << 4), c0, c1, c2);
}

template <typename K>
__global__ void __launch_bounds__(kDetThreads) k_det_reduce(const K* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ off,
                                                            uint32_t m, uint4* __restrict__ tile_sum) {
    __shared__ uint4 tmp[kDetThreads / 32 + 1];
    uint64_t i0 = (uint64_t)blockIdx.x * kDetTile + (uint64_t)threadIdx.x * kDetItems;
    K v[kDetItems + 2];
    load_window(keys, n, i0, v);
    uint4 s = thread_runsum(v, n, i0, off, m);
    uint4 tot;
    block_scan_excl<kDetThreads, false>(s, OpRunSum(), runsum_identity(), tmp, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Exclusive scan over tile summaries; writes per tile (entry state, runs before)
// and the run count r.  One block.
__global__ void __launch_bounds__(1024) k_det_scan(const uint4* __restrict__ tile_sum, uint32_t tiles, uint2* __restrict__ tile_pref,
                                                   uint64_t* __restrict__ counters, uint32_t* __restrict__ run_starts, uint64_t n) {
    __shared__ uint4 tmp[1024 / 32 + 1];
    uint32_t per = (tiles + 1023) / 1024;
    uint32_t b = threadIdx.x * per, e = min(tiles, b + per);
    uint4 acc = runsum_identity();
    OpRunSum op;
    for (uint32_t t = b; t < e; t++) acc = op(acc, tile_sum[t]);
    uint4 tot;
    uint4 pre = block_scan_excl<1024, false>(acc, op, runsum_identity(), tmp, &tot);
    for (uint32_t t = b; t < e; t++) {
        // the state before element 0 is irrelevant (element 0 resets to B); use B
        tile_pref[t] = make_uint2(map_get(pre.x, 0), pre.y);
        pre = op(pre, tile_sum[t]);
    }
    if (threadIdx.x == 0) {
        uint64_t r = tot.y;
        counters[kCtrR] = r;
        run_starts[r] = (uint32_t)n;
    }
}

template <typename K>
__global__ void __launch_bounds__(kDetThreads) k_det_write(const K* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ off,
                                                           uint32_t m, const uint2* __restrict__ tile_pref,
                                                           uint32_t* __restrict__ run_starts, uint8_t* __restrict__ run_desc) {
    __shared__ uint4 tmp[kDetThreads / 32 + 1];
    uint64_t i0 = (uint64_t)blockIdx.x * kDetTile + (uint64_t)threadIdx.x * kDetItems;
    K v[kDetItems + 2];
    load_window(keys, n, i0, v);
    uint4 s = thread_runsum(v, n, i0, off, m);
    uint4 pre = block_scan_excl<kDetThreads, false>(s, OpRunSum(), runsum_identity(), tmp, nullptr);
    uint2 tp = tile_pref[blockIdx.x];
    uint32_t st = map_get(pre.x, tp.x);
    uint32_t cnts[3] = {pre.y, pre.z, pre.w};
    uint32_t idx = tp.y + cnts[tp.x];
    uint64_t nx = next_start(off, m, i0);
#pragma unroll
    for (int j = 0; j < kDetItems; j++) {
        uint64_t i = i0 + j;
        if (i < n) {
            const bool reset = (i == nx);
            if (reset) nx = next_start(off, m, i + 1);
            st = reset ? 0u : step_state(st, v[1 + j] < v[j]);
            if (st == 0) {
                run_starts[idx] = (uint32_t)i;
                // descending iff the next element is in the same array and smaller
                run_desc[idx] = (i + 1 < n && i + 1 != nx && v[2 + j] < v[1 + j]) ? 1 : 0;
                idx++;
            }
        }
    }
}

// Powers of boundaries 1..r-1, sentinels powers[0] = powers[r] = 0, padding
// of 255 up to the next multiple of 32, and the bit set of powers that occur.
__global__ void __launch_bounds__(256) k_powers(const uint32_t* __restrict__ run_starts, const uint64_t* __restrict__ counters,
                                                uint64_t n, uint32_t w, uint64_t magic, uint32_t log2k,
                                                const uint64_t* __restrict__ off, uint32_t m,
                                                const uint2* __restrict__ arr_param,
                                                uint8_t* __restrict__ powers, unsigned long long* __restrict__ level_bits) {
    __shared__ unsigned long long red[256 / 32 + 1];
    __shared__ uint32_t redm[256 / 32 + 1];
    const uint32_t r = (uint32_t)counters[kCtrR];
    unsigned long long bits = 0;
    uint32_t longest = 0;  // longest run seen by this thread
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= r; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t si = run_starts[i];
        uint32_t sp = i >= 1 ? run_starts[i - 1] : 0u;
        longest = max(longest, si - sp);
        // the array holding run i (a batch sorts each array on its own)
        uint64_t base = 0, nn = n;
        uint32_t ww = w;
        uint64_t mg = magic;
        bool arr_start = false;
        if (off != nullptr && i >= 1 && i < r) {
            uint32_t lo = 0, hi = m + 1;  // last a with off[a] <= si
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (off[mid] <= si) lo = mid; else hi = mid;
            }
            base = off[lo];
            nn = off[lo + 1] - base;
            arr_start = (base == si);
            const uint2 prm = arr_param[lo];
            ww = prm.x;
            mg = ((uint64_t)prm.y << 32) | arr_param[m + lo].x;
        }
        const uint64_t d = 2 * nn;
        if (i >= 1 && i < r && !arr_start) {
            uint64_t a2 = (uint64_t)(sp - base) + (si - base);                 // 2n * a
            uint64_t b2 = (uint64_t)(si - base) + (run_starts[i + 1] - base);  // 2n * b
            const uint32_t w = ww;
            const uint64_t magic = mg;
            uint64_t X = a2 << w, Y = b2 << w;
            uint64_t x = __umul64hi(X, magic), y = __umul64hi(Y, magic);
            uint64_t rx = X - x * d, ry = Y - y * d;
            while (rx >= d) { x++; rx -= d; }
            while (ry >= d) { y++; ry -= d; }
            uint32_t h = 63u - (uint32_t)__clzll((long long)(x ^ y));
            uint32_t p2 = w - h;
            uint32_t pk = (p2 + log2k - 1) / log2k;
            powers[i] = (uint8_t)pk;
            bits |= 1ull << pk;
        } else {
            powers[i] = 0;
        }
        if (i == r) {
            uint64_t pad_end = (r + 1 + 31) / 32 * 32;
            for (uint64_t q = r + 1; q < pad_end; q++) powers[q] = 255;
        }
    }
    bits = block_reduce<256>(bits, OpOrU64(), 0ull, red);
    longest = block_reduce<256>(longest, OpMax32(), 0u, redm);
    if (threadIdx.x == 0 && bits) atomicOr(level_bits, bits);
    if (threadIdx.x == 0 && longest)
        atomicMax(reinterpret_cast<unsigned long long*>(const_cast<uint64_t*>(counters) + kCtrMaxRun), (unsigned long long)longest);
}

// Per-array power parameters of a batch: w = ceil(log2 n_a) and the 64-bit
// reciprocal floor((2^64 - 1) / (2 n_a)), stored as prm[a] = (w, magic_hi),
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
        const uint64_t mg = na ? ~0ull / (2 * na) : 0ull;
        prm[a] = make_uint2(w, (uint32_t)(mg >> 32));
        prm[m + a] = make_uint2((uint32_t)mg, 0u);
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

template <typename K>
void launch_detect(const K* keys, uint64_t n, const WsView& ws, cudaStream_t st) {
    uint32_t tiles = (uint32_t)ceil_div(n, kDetTile);
    k_det_reduce<K><<<tiles, kDetThreads, 0, st>>>(keys, n, ws.batch_off, ws.batch_m, ws.det_sum);
    k_det_scan<<<1, 1024, 0, st>>>(ws.det_sum, tiles, ws.det_pref, ws.counters, ws.run_starts, n);
    k_det_write<K><<<tiles, kDetThreads, 0, st>>>(keys, n, ws.batch_off, ws.batch_m, ws.det_pref, ws.run_starts, ws.run_desc);
    g_launches += 3;
}

template void launch_detect<uint32_t>(const uint32_t*, uint64_t, const WsView&, cudaStream_t);
template void launch_detect<uint64_t>(const uint64_t*, uint64_t, const WsView&, cudaStream_t);

void launch_powers(uint64_t n, uint32_t r, int k, const WsView& ws, cudaStream_t st) {
    uint32_t w = 0;
    while ((1ull << w) < n) w++;
    uint64_t magic = ~0ull / (2 * n);
    uint32_t log2k = k == 2 ? 1 : (k == 4 ? 2 : 3);
    uint32_t threads = 256;
    uint32_t blocks = (uint32_t)std::min<uint64_t>(ceil_div((uint64_t)r + 1, threads), 152 * 16);
    if (ws.batch_off) {
        k_array_params<<<(uint32_t)std::min<uint64_t>(ceil_div(ws.batch_m, 256), 1024), 256, 0, st>>>(ws.batch_off, ws.batch_m,
                                                                                                  ws.batch_max_len, ws.batch_prm,
                                                                                                  ws.counters);
        g_launches += 1;
    }
    k_powers<<<blocks, threads, 0, st>>>(ws.run_starts, ws.counters, n, w, magic, log2k, ws.batch_off, ws.batch_m,
                                         ws.batch_prm, ws.powers,
                                          reinterpret_cast<unsigned long long*>(ws.counters + kCtrLevelBits));
    g_launches += 1;
}

}  // namespace mps
