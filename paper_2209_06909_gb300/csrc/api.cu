// api.cu -- C ABI of libmps.so: argument checks, workspace layout and the
// host-side order of the kernels.
//
// Order of one sort (every step is a CUDA kernel; see runs.cu, tree.cu,
// merge.cu):
//   1. run detection (Sec. 2)                       -> run_starts, run_desc
//   2. boundary powers (Def. 3.1)                   -> powers
//   3. min-tree over the powers, depth scans        -> node depths
//   4. node pass (Alg. 1 unrolled)                  -> level nodes, fused subtrees, M
//   5. fused merges of all small subtrees           -> their outputs
//   6. level merges, largest power first            -> root output in keys_out
// The host reads back the run count after step 1 to size steps 2-4, and the
// per-level node counts after step 4 to queue step 6; step 5 takes its count
// from the device and is queued before that second read, so it runs while
// the host waits.  Batches (mps_sort_batch*) read nothing back: every launch
// is sized by bounds and takes its counts from the device.
#include <algorithm>
#include <cstdio>
#include <memory>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mps.h"
#include "common.cuh"
#include "kernels.cuh"

namespace mps {

thread_local uint64_t g_launches = 0;

namespace {

constexpr size_t kAlign = 256;
constexpr uint32_t kMaxMinRun = 32;  // forced runs are sorted by one warp each

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// A device status word as a return code: a bounded wait that ran out is a
// timeout, anything else a failed invariant check.
inline mps_status device_error(uint32_t code) { return code == kDevSpin ? MPS_ERR_TIMEOUT : MPS_ERR_DEVICE_CHECK; }

// Byte layout of the workspace for one (n, key bytes, payload, k).
struct Plan {
    uint64_t n = 0;
    int kb = 4;
    bool vals = false;
    int k = 4;
    MergeGeom g{};
    uint64_t rmax = 0, det_tiles = 0, mask_tiles = 0;
    uint32_t nodes_cap = 0, unit_cap = 0, fused_cap = 0;
    uint64_t lv_cap[kMinTreeLevels] = {};
    int nlv_max = 0;
    // offsets
    size_t o_ctr, o_lvloff, o_det_state, o_rs, o_rdesc, o_fused, o_canon, o_lv[kMinTreeLevels], o_info,
        o_mt, o_nodes_raw, o_nodes_lvl, o_unit_node, o_split, o_udesc, o_ufirst, o_ptiles, o_isz, o_hist, o_tail, o_ktmp, o_vtmp,
        o_incopy, total;

    uint32_t m = 0;  // arrays of a batch (0: a single array)
    size_t o_bprm = 0;
    // minimum run length (1: natural runs) and its buffers
    uint32_t min_run = 1, mr_cap = 0, mr_tiles = 0;
    size_t o_mr_g = 0, o_mr_node = 0, o_mr_tiles = 0, o_mr_desc = 0;

    explicit Plan(uint64_t n_, int kb_, bool vals_, int k_, uint32_t m_ = 0, uint32_t min_run_ = 1, int tile_ = 0)
        : n(n_), kb(kb_), vals(vals_), k(k_), m(m_), min_run(min_run_) {
        g = merge_geom(kb, vals, k, tile_);
        rmax = n / 2 + m + 2;
        det_tiles = ceil_div(std::max<uint64_t>(n, 1), kDetTile);
        mask_tiles = ceil_div(rmax, kMaskTile);
        nodes_cap = (uint32_t)(34 * (n / g.tmax + 1) + 64);
        unit_cap = (uint32_t)(n / g.ts + n / g.tmax + 64);
        // fused subtrees: at most k children of each node above T_max, plus one
        // root per array (a single array, or every array of a batch)
        fused_cap = (uint32_t)k * nodes_cap + std::max<uint32_t>(m, 1) + 64;
        uint64_t len = rmax + 1;
        nlv_max = 0;
        while (true) {
            lv_cap[nlv_max] = (len + 31) / 32 * 32 + 32;
            nlv_max++;
            if (len <= 32 || nlv_max == kMinTreeLevels) break;
            len = ceil_div(len, 32);
        }
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t at = o; o += align_up(bytes); return at; };
        o_ctr = take(kCtrWords * 8);
        o_lvloff = take(kMaxLevels * 4);
        o_det_state = take(det_tiles * 24 + (ceil_div(std::max<uint64_t>(n, 1), 32) + 8) * 4);
        o_rs = take((rmax + 2 + 32) * 4);  // padded for 16-byte loads past r
        o_rdesc = take(rmax + 1);
        o_fused = take((size_t)fused_cap * 16);
        o_canon = take((rmax + 1) * 4);
        for (int t = 0; t < kMinTreeLevels; t++) o_lv[t] = t < nlv_max ? take(lv_cap[t]) : 0;
        o_info = take(rmax + 1 + 16);
        o_mt = take(mask_tiles * 8 * 4);
        o_nodes_raw = take((size_t)nodes_cap * sizeof(LevelNode));
        o_nodes_lvl = take((size_t)nodes_cap * sizeof(LevelNode));
        o_unit_node = take((size_t)unit_cap * 4);
        o_split = take((size_t)(unit_cap + 1) * k * 4);
        o_udesc = take((size_t)unit_cap * kUnitDescBytes);
        o_ufirst = take((size_t)unit_cap * 4);
        o_ptiles = take((size_t)(unit_cap / kPackTile + 2) * 4);
        o_isz = take((size_t)(unit_cap + 64) * 4);  // padded for 16-byte loads past the last interval
        o_hist = take(mask_tiles * kMaxLevels * 4);
        o_tail = take(kTailCap * 4);
        o_bprm = take((size_t)2 * std::max<uint32_t>(m, 1) * 8);
        o_ktmp = take(n * kb);
        o_vtmp = vals ? take(n * 4) : o;
        // a single array may be sorted into the memory it is read from: room for a copy of the input
        o_incopy = m == 0 ? take(n * kb) : o;
        if (m == 0 && vals) take(n * 4);
        if (min_run > 1) {
            // good intervals: natural runs with >= min_run - 1 interior flags, at most n / (min_run - 1) + 1
            mr_cap = (uint32_t)(n / (min_run - 1) + 2);
            mr_tiles = (uint32_t)(ceil_div(std::max<uint64_t>(rmax, (uint64_t)mr_cap + 2), 4096) + 2);
            o_mr_g = take((size_t)3 * mr_cap * 4);
            o_mr_node = take((size_t)7 * (mr_cap + 2) * 4);
            o_mr_tiles = take((size_t)mr_tiles * 4);
            o_mr_desc = take(rmax + 1);
        }
        total = o;
    }

    MinRunView min_run_view(void* base) const {
        char* b = static_cast<char*>(base);
        MinRunView v{};
        v.m = min_run;
        v.cap = mr_cap;
        uint32_t* g = reinterpret_cast<uint32_t*>(b + o_mr_g);
        v.gs = g;
        v.ge = g + mr_cap;
        v.gv = g + 2 * (size_t)mr_cap;
        uint32_t* nd = reinterpret_cast<uint32_t*>(b + o_mr_node);
        const size_t nn = (size_t)mr_cap + 2;
        v.succ = nd;
        v.hit = nd + nn;
        v.cnt = nd + 2 * nn;
        v.off = nd + 3 * nn;
        v.mark = nd + 4 * nn;
        v.jmp0 = nd + 5 * nn;
        v.jmp1 = nd + 6 * nn;
        v.tiles = reinterpret_cast<uint32_t*>(b + o_mr_tiles);
        v.tiles_cap = mr_tiles;
        v.desc_nat = reinterpret_cast<uint8_t*>(b + o_mr_desc);
        return v;
    }

    WsView view(void* base) const {
        char* b = static_cast<char*>(base);
        WsView w{};
        w.n = n;
        w.counters = reinterpret_cast<uint64_t*>(b + o_ctr);
        w.det_state = reinterpret_cast<uint64_t*>(b + o_det_state);
        w.run_starts = reinterpret_cast<uint32_t*>(b + o_rs);
        w.run_desc = reinterpret_cast<uint8_t*>(b + o_rdesc);
        w.fused_list = reinterpret_cast<uint4*>(b + o_fused);
        w.fused_cap = fused_cap;
        for (int t = 0; t < kMinTreeLevels; t++) w.lv[t] = t < nlv_max ? reinterpret_cast<uint8_t*>(b + o_lv[t]) : nullptr;
        w.powers = w.lv[0];
        w.node_info = reinterpret_cast<uint8_t*>(b + o_info);
        unsigned long long* mt = reinterpret_cast<unsigned long long*>(b + o_mt);
        w.mt_f = mt;
        w.mt_g = mt + mask_tiles;
        w.mt_fpre = mt + 2 * mask_tiles;
        w.mt_gsuf = mt + 3 * mask_tiles;
        w.level_off = reinterpret_cast<uint32_t*>(b + o_lvloff);
        w.nodes_raw = reinterpret_cast<LevelNode*>(b + o_nodes_raw);
        w.nodes_lvl = reinterpret_cast<LevelNode*>(b + o_nodes_lvl);
        w.nodes_cap = nodes_cap;
        w.unit_node = reinterpret_cast<uint32_t*>(b + o_unit_node);
        w.split_tab = reinterpret_cast<uint32_t*>(b + o_split);
        w.unit_desc = b + o_udesc;
        w.unit_first = reinterpret_cast<uint32_t*>(b + o_ufirst);
        w.pack_tiles = reinterpret_cast<uint32_t*>(b + o_ptiles);
        w.ivl_size = reinterpret_cast<uint32_t*>(b + o_isz);
        w.unit_cap = unit_cap;
        w.canon_idx = reinterpret_cast<uint32_t*>(b + o_canon);
        w.cand_cap = (uint32_t)(rmax + 1);
        w.hist = reinterpret_cast<uint32_t*>(b + o_hist);
        w.tail_list = reinterpret_cast<uint32_t*>(b + o_tail);
        w.keys_tmp = b + o_ktmp;
        w.vals_tmp = vals ? reinterpret_cast<uint32_t*>(b + o_vtmp) : nullptr;
        w.batch_off = nullptr;
        w.batch_m = 0;
        w.batch_max_len = 0;
        w.batch_cost = nullptr;
        w.batch_prm = reinterpret_cast<uint2*>(b + o_bprm);
        return w;
    }
};

// Sets the min-tree level lengths for the actual run count.
void set_levels(WsView& w, uint32_t r) {
    uint64_t len = (uint64_t)r + 1;
    int nl = 0;
    while (true) {
        w.lv_len[nl] = (uint32_t)len;
        nl++;
        if (len <= 32 || nl == kMinTreeLevels) break;
        len = ceil_div(len, 32);
    }
    w.nlv = nl;
}

// ------------------------------------------------------------- profiling

// Algorithmic bytes of a profiled stage.  Some are known when the stage is
// queued; the others depend on device counters (the run count, the merge
// cost and the per-level node sizes) and are computed from a snapshot of the
// sort's counter block, copied to pinned host memory behind the sort's last
// kernel, when mps_profile_read asks for them.
enum ByteRule : int {
    kBytesFixed = 0,   // `bytes` as given
    kBytesFused = 1,   // 2 * b * (M - elements merged by level merges), b = `bytes`
    kBytesLevel = 2,   // 2 * b * (elements of the nodes of power p), b = `bytes`
    kBytesPerRun = 3,  // `bytes` * r
};

struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
    double bytes;
    int rule;
    int p;
    int snap;  // counter snapshot of the sort the stage belongs to (-1: none)
};

constexpr int kSnapSlots = 256;
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;
uint64_t* g_snap_host = nullptr;  // kSnapSlots counter blocks, pinned
cudaEvent_t g_snap_ev[kSnapSlots];
int g_snap_used = 0;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// One stage of a sort: an NVTX range of the stage's name around the host
// code that queues it (always; NVTX does nothing unless a tracer attaches),
// and, while mps_profile_enable is on, CUDA events on the stream around its
// kernels.
struct ProfScope {
    bool on;
    ProfRec rec;
    cudaStream_t st;
    ProfScope(const char* name, double bytes, cudaStream_t s, int rule = kBytesFixed, int p = 0) : on(false), st(s) {
        nvtxRangePushA(name);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_on) return;
        on = true;
        rec.name = name;
        rec.bytes = bytes;
        rec.rule = rule;
        rec.p = p;
        rec.snap = -1;
        rec.a = take_event();
        rec.b = take_event();
        cudaEventRecord(rec.a, st);
    }
    ~ProfScope() {
        nvtxRangePop();
        if (!on) return;
        cudaEventRecord(rec.b, st);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back(rec);
    }
};

size_t prof_mark() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof.size();
}

// Behind the last kernel of a sort: a copy of its counter block for the
// stages recorded since `mark` (only while profiling).
void prof_snapshot(size_t mark, const uint64_t* d_ctr, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on || g_prof.size() <= mark || !g_snap_host || g_snap_used >= kSnapSlots) return;
    const int slot = g_snap_used++;
    if (cudaMemcpyAsync(g_snap_host + (size_t)slot * kCtrWords, d_ctr, kCtrWords * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return;
    cudaEventRecord(g_snap_ev[slot], st);
    for (size_t i = mark; i < g_prof.size(); i++) g_prof[i].snap = slot;
}

// elements merged by level merges (nodes above the fused-tile size), from a counter block
uint64_t level_elems(const uint64_t* h) {
    uint64_t s = 0;
    for (int p = 1; p < kMaxLevels; p++) s += h[kCtrHbmCount + p] ? h[kCtrHbmSize + p] : 0;
    return s;
}

double rec_bytes(const ProfRec& r) {
    if (r.rule == kBytesFixed) return r.bytes;
    if (r.snap < 0) return 0.0;
    cudaEventSynchronize(g_snap_ev[r.snap]);
    const uint64_t* h = g_snap_host + (size_t)r.snap * kCtrWords;
    switch (r.rule) {
        case kBytesFused: {
            const uint64_t lv = level_elems(h);
            return 2.0 * r.bytes * (double)(h[kCtrM] >= lv ? h[kCtrM] - lv : 0);
        }
        case kBytesLevel: return h[kCtrHbmCount + r.p] ? 2.0 * r.bytes * (double)h[kCtrHbmSize + r.p] : 0.0;
        case kBytesPerRun: return r.bytes * (double)h[kCtrR];
    }
    return 0.0;
}

// ------------------------------------------------------------- statistics

// The most recent sort on this host thread: its statistics live in its
// workspace's counter block and are read back (after synchronising its
// stream) only when mps_last_stats asks for them.
struct LastSort {
    const uint64_t* d_ctr = nullptr;
    cudaStream_t st = nullptr;
    double b = 4.0;           // bytes per element (key + payload)
    bool pending = false;     // counters not read back yet
};
thread_local LastSort g_pending;
thread_local mps_stats g_last{};

void stats_from_counters(const uint64_t* h, double b, mps_stats& s) {
    s.r = h[kCtrR];
    s.merge_cost = h[kCtrM];
    s.frontier_nodes = h[kCtrFrontier];
    s.hbm_nodes = h[kCtrHbmTotal];
    s.num_levels = (uint32_t)__builtin_popcountll(h[kCtrLevelBits]);
    s.device_status = (uint32_t)h[kCtrStatus];
    s.hbm_levels = 0;
    for (int p = 1; p < kMaxLevels; p++) s.hbm_levels += h[kCtrHbmCount + p] ? 1u : 0u;
    const uint64_t lv = level_elems(h);
    s.bytes_levels = (uint64_t)(2.0 * b * (double)lv);
    s.bytes_fused = (uint64_t)(2.0 * b * (double)(s.merge_cost >= lv ? s.merge_cost - lv : 0));
}

// Synchronises the pending sort's stream and fills g_last from its counters.
mps_status settle_last() {
    if (!g_pending.pending) return MPS_OK;
    g_pending.pending = false;
    uint64_t h[kCtrWords];
    if (cudaMemcpyAsync(h, g_pending.d_ctr, sizeof(h), cudaMemcpyDeviceToHost, g_pending.st) != cudaSuccess ||
        cudaStreamSynchronize(g_pending.st) != cudaSuccess)
        return MPS_ERR_CUDA;
    stats_from_counters(h, g_pending.b, g_last);
    return MPS_OK;
}

bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
    if (!a || !b || !an || !bn) return false;
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bn && y < x + an;
}

#define MPS_CUDA(call)                                 \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return MPS_ERR_CUDA;    \
    } while (0)

// Largest power whose nodes can be larger than a fused tile (T_max elements)
// in arrays of at most max_len elements.  Every boundary inside a node of
// power v has power >= v, i.e. the normalised midpoints of adjacent runs agree
// on their first (v-1) log2 k bits (Def. 3.1 with P_k = ceil(P_2 / log2 k)):
// all run midpoints of the node lie in one interval of max_len / k^(v-1)
// elements.  Its first and last runs each meet a boundary of power >= v, so
// each is shorter than 2 max_len / k^(v-1).  The node is therefore smaller
// than 3 max_len / k^(v-1), and level merges exist only for powers v with
// T_max k^(v-1) < 3 max_len; the bound below uses 4 max_len as margin.
// Bound on the largest power of any boundary of an array of n elements:
// P_k <= ceil(log_k n + 1) (Sec. 3.3), plus one as margin.
int max_power_bound(uint64_t n, int k) {
    int lg = 0;
    while ((1ull << lg) < std::max<uint64_t>(n, 1)) lg++;
    const int t = __builtin_ctz((unsigned)k);
    return (lg + t - 1) / t + 2;
}

// Tile choice of a single-array sort: the default, except uint32 keys with a
// minimum run length, whose extended runs favour the larger fused tile (one
// level merge fewer; measured on the 2^28 permutation with m = 24).
int single_tile(int kb, bool vals, uint32_t min_run) { return (min_run > 1 && kb == 4 && !vals) ? 1 : 0; }

int level_power_bound(uint64_t max_len, int k, uint32_t tmax) {
    const uint64_t lim = 4 * std::max<uint64_t>(max_len, 1);
    uint64_t span = tmax;  // T_max * k^(v-1)
    int v = 0;
    while (span < lim && v < kMaxLevels - 1) {
        v++;
        span *= (uint64_t)k;
    }
    return v;
}

// One array: every launch is sized by bounds from n and takes its counts from
// the device, so the call only queues kernels on the stream and returns; no
// host thread waits for the device.  Levels are queued for every power up to
// the bound for n; a level without nodes costs its launches and nothing else.
template <typename K, bool V>
mps_status sort_impl(const K* keys_in, const uint32_t* vals_in, K* keys_out, uint32_t* vals_out, uint64_t n, int k,
                     void* d_ws, size_t ws_bytes, const mps_tree* tree, bool move_keys, cudaStream_t st,
                     uint32_t min_run = 1, int tail = 0) {
    if (!fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (min_run < 1 || min_run > kMaxMinRun) return MPS_ERR_UNSUPPORTED;
    if (tail < 0 || tail > 2) return MPS_ERR_INVALID_ARG;
    // for k = 2 every final-collapse node has one boundary: all policies build the same tree
    const bool relabel = tail != 0 && k > 2;
    // run starts are 32-bit positions; a minimum run length steps positions by
    // m, which is kept clear of wrapping by the lower limit
    if (n >= (1ull << 32) || (min_run > 1 && n >= (1ull << 31))) return MPS_ERR_UNSUPPORTED;
    const double b = (double)sizeof(K) + (V ? 4.0 : 0.0);
    g_launches = 0;
    if (n == 0) {
        if (tree && tree->counts) MPS_CUDA(cudaMemsetAsync(tree->counts, 0, 4 * sizeof(uint64_t), st));
        g_pending.pending = false;
        g_last = mps_stats{};
        return MPS_OK;
    }
    if (!keys_in || !d_ws) return MPS_ERR_INVALID_ARG;
    if (move_keys && !keys_out) return MPS_ERR_INVALID_ARG;
    if (tree && tree->nodes && !tree->node_first) return MPS_ERR_INVALID_ARG;  // the node table needs node_first
    if (V && move_keys && (!vals_in || !vals_out)) return MPS_ERR_INVALID_ARG;
    const size_t kbytes = n * sizeof(K), vbytes = n * 4;
    // keys and payloads must not overlap each other (an output may overlap its own input)
    if (V && move_keys &&
        (overlaps(keys_in, kbytes, vals_out, vbytes) || overlaps(vals_in, vbytes, keys_out, kbytes) ||
         overlaps(keys_out, kbytes, vals_out, vbytes)))
        return MPS_ERR_INVALID_ARG;
    Plan plan(n, sizeof(K), V, k, 0, min_run, single_tile((int)sizeof(K), V, min_run));
    if (ws_bytes < plan.total) return MPS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(d_ws) % 16) return MPS_ERR_INVALID_ARG;
    WsView ws = plan.view(d_ws);
    const MergeGeom& g = plan.g;
    const size_t mark = prof_mark();
    const K* keys_orig = keys_in;

    MPS_CUDA(cudaMemsetAsync(ws.counters, 0, kCtrWords * 8, st));
    // The merges read leaves from the input while node outputs land in
    // keys_out, so an output that overlaps its input sorts a copy of the input
    // (kept in the workspace).
    // A minimum run length sorts its short runs in the same copy.
    if (min_run > 1 ||
        (move_keys && (overlaps(keys_in, kbytes, keys_out, kbytes) || (V && overlaps(vals_in, vbytes, vals_out, vbytes))))) {
        K* kc = reinterpret_cast<K*>(static_cast<char*>(d_ws) + plan.o_incopy);
        MPS_CUDA(cudaMemcpyAsync(kc, keys_in, kbytes, cudaMemcpyDeviceToDevice, st));
        keys_in = kc;
        if (V) {
            uint32_t* vc = reinterpret_cast<uint32_t*>(static_cast<char*>(d_ws) + plan.o_incopy + align_up(kbytes));
            MPS_CUDA(cudaMemcpyAsync(vc, vals_in, vbytes, cudaMemcpyDeviceToDevice, st));
            vals_in = vc;
        }
    }
    const uint32_t r_bound = (uint32_t)std::min<uint64_t>(plan.rmax, n + 1);
    set_levels(ws, r_bound);
    {
        ProfScope ps("detect_runs", (double)kbytes, st);
        launch_detect<K>(keys_orig, n, ws, st);
    }
    if (min_run > 1) {
        // natural runs -> runs of at least min_run elements, the short ones sorted in the copy
        ProfScope ps("min_run", 2.0 * (double)kbytes, st);
        launch_min_run<K, V>(keys_orig, const_cast<K*>(keys_in), const_cast<uint32_t*>(vals_in), n,
                             plan.min_run_view(d_ws), ws, st);
    }
    if (move_keys) {
        ProfScope ps("copy_single_run", 0.0, st);
        launch_copy_single_run<K, V>(keys_in, vals_in, keys_out, vals_out, n, ws, st);
    }
    {
        ProfScope ps("powers", 9.0, st, kBytesPerRun);
        launch_powers(n, r_bound, k, ws, st);
    }
    if (relabel) {
        // the stack's final collapse by count: relabelled powers, original ones to the tree output
        ProfScope ps("tail_relabel", 0.0, st);
        launch_tail(r_bound, k, tail, tree ? tree->powers : nullptr, ws, st);
    }
    {
        ProfScope ps("tree_scans", 4.0, st, kBytesPerRun);
        launch_mintree(r_bound, ws, st);
        launch_masks(r_bound, tree && tree->leaf_depth, tree ? tree->leaf_depth : nullptr, n, k, g.tmax, ws, st);
    }
    {
        ProfScope ps("node_pass", 2.0, st, kBytesPerRun);
        launch_node_pass(r_bound, k, g.tmax, (uint32_t)level_power_bound(n, k, g.tmax), ws, st);
    }
    if (move_keys) {
        launch_bucket(plan.nodes_cap, ws, st);
        {
            // algorithmic bytes (Sec. 2.2 cost model): one read and one write of
            // b bytes per element per merge inside the fused subtrees
            ProfScope ps("fused_merge", b, st, kBytesFused);
            launch_fused<K, V>(keys_in, vals_in, keys_out, vals_out, plan.fused_cap, g, ws, st);
        }
        const uint32_t nn_bound = (uint32_t)(n / g.tmax + 1);
        // relabelled powers rise by the number of final-collapse nodes, at most the largest power
        const int ptop = level_power_bound(n, k, g.tmax) + (relabel ? max_power_bound(n, k) : 0);
        for (int p = ptop; p >= 1; p--) {
            {
                ProfScope ps("level_plan", 0.0, st);
                launch_level_plan<K>(p, nn_bound, n, k, keys_in, keys_out, g, ws, st);
            }
            ProfScope ps("level_merge", b, st, kBytesLevel, p);
            launch_level_merge<K, V>(nn_bound, n, keys_in, vals_in, keys_out, vals_out, g, ws, st);
        }
    }
    if (tree) {
        if (tree->run_starts || tree->run_desc || tree->powers || tree->leaf_depth || tree->counts)
            launch_tree_arrays(r_bound, ws, min_run > 1 ? plan.min_run_view(d_ws).desc_nat : ws.run_desc, tree->run_starts,
                               tree->run_desc, relabel ? nullptr : tree->powers, tree->leaf_depth, tree->counts, st);
        if (tree->node_first) launch_tree_dump(r_bound, k, ws, tree->node_first, tree->nodes, st);
    }
    MPS_CUDA(cudaGetLastError());
    prof_snapshot(mark, ws.counters, st);
    g_last = mps_stats{};
    g_last.n = n;
    g_last.launches = g_launches;
    g_pending.d_ctr = ws.counters;
    g_pending.st = st;
    g_pending.b = b;
    g_pending.pending = true;
    return MPS_OK;
}

// Batch of m arrays laid end to end (offsets d_off[0..m], d_off[m] = n).
// Every launch takes its counts from device counters, so the sequence makes
// no host synchronisation until the optional final status check and can be
// captured into a CUDA graph.
template <typename K, bool V>
mps_status batch_impl(const K* keys_in, const uint32_t* vals_in, K* keys_out, uint32_t* vals_out, uint64_t n,
                      const uint64_t* d_off, uint32_t m, uint64_t max_len, int k, void* d_ws, size_t ws_bytes,
                      uint64_t* d_costs, bool sync_at_end, cudaStream_t st, int tile) {
    if (!fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (tile < 0 || tile >= kTileChoices) return MPS_ERR_INVALID_ARG;
    if (n >= (1ull << 32)) return MPS_ERR_UNSUPPORTED;
    struct Range {  // NVTX range around the whole batch
        Range() { nvtxRangePushA("sort_batch"); }
        ~Range() { nvtxRangePop(); }
    } range;
    if (d_costs && m) MPS_CUDA(cudaMemsetAsync(d_costs, 0, (size_t)m * 8, st));
    if (n == 0) return MPS_OK;
    if (!keys_in || !keys_out || !d_off || !d_ws || m == 0) return MPS_ERR_INVALID_ARG;
    if (V && (!vals_in || !vals_out)) return MPS_ERR_INVALID_ARG;
    if (overlaps(keys_in, n * sizeof(K), keys_out, n * sizeof(K))) return MPS_ERR_INVALID_ARG;
    if (V && overlaps(vals_in, n * 4, vals_out, n * 4)) return MPS_ERR_INVALID_ARG;
    Plan plan(n, sizeof(K), V, k, m, 1, tile);
    if (ws_bytes < plan.total) return MPS_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(d_ws) % 16) return MPS_ERR_INVALID_ARG;
    WsView ws = plan.view(d_ws);
    ws.batch_off = d_off;
    ws.batch_m = m;
    ws.batch_max_len = max_len;
    ws.batch_cost = d_costs;
    const MergeGeom& g = plan.g;
    g_launches = 0;
    const uint32_t r_bound = (uint32_t)std::min<uint64_t>(plan.rmax, n + 1);
    set_levels(ws, r_bound);
    MPS_CUDA(cudaMemsetAsync(ws.counters, 0, kCtrWords * 8, st));
    launch_detect<K>(keys_in, n, ws, st);
    launch_powers(n, r_bound, k, ws, st);
    launch_mintree(r_bound, ws, st);
    launch_masks(r_bound, false, nullptr, n, k, g.tmax, ws, st);
    launch_node_pass(r_bound, k, g.tmax, (uint32_t)level_power_bound(max_len ? max_len : n, k, g.tmax), ws, st);
    launch_copy_lone_runs<K, V>(keys_in, vals_in, keys_out, vals_out, r_bound, ws, st);
    launch_bucket(plan.nodes_cap, ws, st);
    launch_fused<K, V>(keys_in, vals_in, keys_out, vals_out, plan.fused_cap, g, ws, st);
    const uint32_t nn_bound = (uint32_t)(n / g.tmax + 1);
    for (int p = level_power_bound(max_len ? max_len : n, k, g.tmax); p >= 1; p--) {
        launch_level_plan<K>(p, nn_bound, n, k, keys_in, keys_out, g, ws, st);
        launch_level_merge<K, V>(nn_bound, n, keys_in, vals_in, keys_out, vals_out, g, ws, st);
    }
    MPS_CUDA(cudaGetLastError());
    g_pending.pending = false;
    if (sync_at_end) {
        uint64_t h_ctr[kCtrWords];
        MPS_CUDA(cudaMemcpyAsync(h_ctr, ws.counters, sizeof(h_ctr), cudaMemcpyDeviceToHost, st));
        MPS_CUDA(cudaStreamSynchronize(st));
        g_last = mps_stats{};
        g_last.n = n;
        stats_from_counters(h_ctr, (double)sizeof(K) + (V ? 4.0 : 0.0), g_last);
        g_last.launches = g_launches;
        if ((uint32_t)h_ctr[kCtrStatus]) return device_error((uint32_t)h_ctr[kCtrStatus]);
    }
    return MPS_OK;
}

}  // namespace
}  // namespace mps

using namespace mps;

extern "C" {

mps_status mps_workspace_size(uint64_t n, mps_key_type kt, int has_payload, int k, size_t* bytes) {
    if (!bytes) return MPS_ERR_INVALID_ARG;
    if (kt != MPS_U32 && kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    if (!fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (n >= (1ull << 32)) return MPS_ERR_UNSUPPORTED;
    Plan p(n, kt == MPS_U32 ? 4 : 8, has_payload != 0, k);
    *bytes = p.total;
    return MPS_OK;
}

mps_status mps_sort_keys(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k, void* d_ws,
                         size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream) {
    if (kt == MPS_U32)
        return sort_impl<uint32_t, false>((const uint32_t*)d_keys_in, nullptr, (uint32_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, false>((const uint64_t*)d_keys_in, nullptr, (uint64_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_sort_pairs(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out, uint32_t* d_vals_out,
                          uint64_t n, mps_key_type kt, int k, void* d_ws, size_t ws_bytes, const mps_tree* opt_tree,
                          cudaStream_t stream) {
    if (kt == MPS_U32)
        return sort_impl<uint32_t, true>((const uint32_t*)d_keys_in, d_vals_in, (uint32_t*)d_keys_out, d_vals_out, n, k, d_ws,
                                         ws_bytes, opt_tree, true, stream);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, true>((const uint64_t*)d_keys_in, d_vals_in, (uint64_t*)d_keys_out, d_vals_out, n, k, d_ws,
                                         ws_bytes, opt_tree, true, stream);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_merge_tree(const void* d_keys, uint64_t n, mps_key_type kt, int k, const mps_tree* out, void* d_ws,
                          size_t ws_bytes, cudaStream_t stream) {
    if (!out) return MPS_ERR_INVALID_ARG;
    if (kt == MPS_U32)
        return sort_impl<uint32_t, false>((const uint32_t*)d_keys, nullptr, nullptr, nullptr, n, k, d_ws, ws_bytes, out, false,
                                          stream);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, false>((const uint64_t*)d_keys, nullptr, nullptr, nullptr, n, k, d_ws, ws_bytes, out, false,
                                          stream);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_workspace_size_minrun(uint64_t n, mps_key_type kt, int has_payload, int k, uint32_t min_run_len,
                                     size_t* bytes) {
    if (!bytes) return MPS_ERR_INVALID_ARG;
    if (kt != MPS_U32 && kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    if (!fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (n >= (1ull << 31) || min_run_len < 1 || min_run_len > kMaxMinRun) return MPS_ERR_UNSUPPORTED;
    Plan p(n, kt == MPS_U32 ? 4 : 8, has_payload != 0, k, 0, min_run_len,
           single_tile(kt == MPS_U32 ? 4 : 8, has_payload != 0, min_run_len));
    *bytes = p.total;
    return MPS_OK;
}

mps_status mps_sort_keys_minrun(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k,
                                uint32_t min_run_len, void* d_ws, size_t ws_bytes, const mps_tree* opt_tree,
                                cudaStream_t stream) {
    if (kt == MPS_U32)
        return sort_impl<uint32_t, false>((const uint32_t*)d_keys_in, nullptr, (uint32_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream, min_run_len);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, false>((const uint64_t*)d_keys_in, nullptr, (uint64_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream, min_run_len);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_sort_keys_tail(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k, int tail_policy,
                              void* d_ws, size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream) {
    if (kt == MPS_U32)
        return sort_impl<uint32_t, false>((const uint32_t*)d_keys_in, nullptr, (uint32_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream, 1u, tail_policy);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, false>((const uint64_t*)d_keys_in, nullptr, (uint64_t*)d_keys_out, nullptr, n, k, d_ws,
                                          ws_bytes, opt_tree, true, stream, 1u, tail_policy);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_sort_pairs_minrun(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out, uint32_t* d_vals_out,
                                 uint64_t n, mps_key_type kt, int k, uint32_t min_run_len, void* d_ws, size_t ws_bytes,
                                 const mps_tree* opt_tree, cudaStream_t stream) {
    if (kt == MPS_U32)
        return sort_impl<uint32_t, true>((const uint32_t*)d_keys_in, d_vals_in, (uint32_t*)d_keys_out, d_vals_out, n, k, d_ws,
                                         ws_bytes, opt_tree, true, stream, min_run_len);
    if (kt == MPS_U64)
        return sort_impl<uint64_t, true>((const uint64_t*)d_keys_in, d_vals_in, (uint64_t*)d_keys_out, d_vals_out, n, k, d_ws,
                                         ws_bytes, opt_tree, true, stream, min_run_len);
    return MPS_ERR_INVALID_ARG;
}

mps_status mps_sort_keys_host_async(const void* h_keys_in, void* h_keys_out, uint64_t n, mps_key_type kt, int k,
                                    void* d_keys_in, void* d_keys_out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (n && (!h_keys_in || !h_keys_out || !d_keys_in || !d_keys_out)) return MPS_ERR_INVALID_ARG;
    // the sort's argument checks, made before the input copy is queued, so that
    // a rejected call leaves nothing in flight
    size_t need = 0;
    const mps_status sz = mps_workspace_size(n, kt, 0, k, &need);
    if (sz != MPS_OK) return sz;
    if (n && (!d_ws || reinterpret_cast<uintptr_t>(d_ws) % 16)) return MPS_ERR_INVALID_ARG;
    if (n && ws_bytes < need) return MPS_ERR_WORKSPACE;
    const size_t bytes = n * (kt == MPS_U32 ? 4 : 8);
    if (n && cudaMemcpyAsync(d_keys_in, h_keys_in, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) return MPS_ERR_CUDA;
    mps_status s = mps_sort_keys(d_keys_in, d_keys_out, n, kt, k, d_ws, ws_bytes, nullptr, stream);
    if (s != MPS_OK) return s;
    if (n && cudaMemcpyAsync(h_keys_out, d_keys_out, bytes, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return MPS_ERR_CUDA;
    return MPS_OK;
}

mps_status mps_sort_keys_host(const void* h_keys_in, void* h_keys_out, uint64_t n, mps_key_type kt, int k, void* d_keys_in,
                              void* d_keys_out, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    mps_status s = mps_sort_keys_host_async(h_keys_in, h_keys_out, n, kt, k, d_keys_in, d_keys_out, d_ws, ws_bytes, stream);
    if (s != MPS_OK) return s;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return MPS_ERR_CUDA;
    return MPS_OK;
}

}  // extern "C"

// ------------------------------------------------------------- batches

namespace mps {
namespace {

std::mutex g_tune_mu;
// Batch configuration chosen by k = 0: fan-in and tile choice per key type,
// payload flag and log2 of the mean array size (k = 0: not tuned).
struct TunedCfg {
    int k = 0, tile = 0;
};
TunedCfg g_tuned[2][2][64];

int size_bucket(uint64_t n, uint32_t m) {
    const uint64_t mean = m ? n / m : n;
    int b = 0;
    while ((1ull << (b + 1)) <= std::max<uint64_t>(mean, 1) && b < 63) b++;
    return b;
}

TunedCfg tuned_cfg(mps_key_type kt, bool vals, uint64_t n, uint32_t m) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TunedCfg c = g_tuned[kt == MPS_U64][vals][size_bucket(n, m)];
    if (!c.k) c = TunedCfg{4, 0};
    return c;
}

void set_tuned_cfg(mps_key_type kt, bool vals, uint64_t n, uint32_t m, TunedCfg c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[kt == MPS_U64][vals][size_bucket(n, m)] = c;
}

}  // namespace

mps_status batch_dispatch(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out, uint64_t n,
                          const uint64_t* d_off, uint32_t m, uint64_t max_len, mps_key_type kt, int k, void* d_ws,
                          size_t ws_bytes, uint64_t* d_costs, bool sync_at_end, cudaStream_t st, int tile) {
    const bool vals = vals_in != nullptr || vals_out != nullptr;
    if (k == 0) {
        const TunedCfg c = tuned_cfg(kt, vals, n, m);
        k = c.k;
        tile = c.tile;
    }
    if (kt == MPS_U32) {
        if (vals)
            return batch_impl<uint32_t, true>((const uint32_t*)keys_in, vals_in, (uint32_t*)keys_out, vals_out, n, d_off, m,
                                              max_len, k, d_ws, ws_bytes, d_costs, sync_at_end, st, tile);
        return batch_impl<uint32_t, false>((const uint32_t*)keys_in, nullptr, (uint32_t*)keys_out, nullptr, n, d_off, m,
                                           max_len, k, d_ws, ws_bytes, d_costs, sync_at_end, st, tile);
    }
    if (kt == MPS_U64) {
        if (vals)
            return batch_impl<uint64_t, true>((const uint64_t*)keys_in, vals_in, (uint64_t*)keys_out, vals_out, n, d_off, m,
                                              max_len, k, d_ws, ws_bytes, d_costs, sync_at_end, st, tile);
        return batch_impl<uint64_t, false>((const uint64_t*)keys_in, nullptr, (uint64_t*)keys_out, nullptr, n, d_off, m,
                                           max_len, k, d_ws, ws_bytes, d_costs, sync_at_end, st, tile);
    }
    return MPS_ERR_INVALID_ARG;
}

}  // namespace mps

struct mps_batch_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t* counters = nullptr;  // device counter block of the captured workspace
};

extern "C" {

mps_status mps_batch_workspace_size(uint64_t n, uint32_t m, mps_key_type kt, int has_payload, int k, size_t* bytes) {
    if (!bytes) return MPS_ERR_INVALID_ARG;
    if (kt != MPS_U32 && kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    if (k != 0 && !fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (n >= (1ull << 32)) return MPS_ERR_UNSUPPORTED;
    // k = 0 (the tuned configuration): the largest over fan-ins 2, 4, 8 (and 16
    // if set by mps_batch_set_config) and every tile choice
    size_t best = 0;
    for (int kk : {2, 4, 8, 16}) {
        if (k != 0 && kk != k) continue;
        for (int tile = 0; tile < kTileChoices; tile++) {
            if (k != 0 && tile != 0) continue;
            Plan p(n, kt == MPS_U32 ? 4 : 8, has_payload != 0, kk, m, 1, tile);
            best = std::max(best, p.total);
        }
    }
    *bytes = best;
    return MPS_OK;
}

mps_status mps_sort_batch(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m, uint64_t n,
                          uint64_t max_len, mps_key_type kt, int k, void* d_ws, size_t ws_bytes, uint64_t* d_merge_costs,
                          cudaStream_t stream) {
    return batch_dispatch(d_keys_in, nullptr, d_keys_out, nullptr, n, d_offsets, m, max_len, kt, k, d_ws, ws_bytes,
                          d_merge_costs, true, stream, 0);
}

mps_status mps_sort_batch_pairs(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out, uint32_t* d_vals_out,
                                const uint64_t* d_offsets, uint32_t m, uint64_t n, uint64_t max_len, mps_key_type kt, int k,
                                void* d_ws, size_t ws_bytes, uint64_t* d_merge_costs, cudaStream_t stream) {
    if (!d_vals_in || !d_vals_out) return n ? MPS_ERR_INVALID_ARG : MPS_OK;
    return batch_dispatch(d_keys_in, d_vals_in, d_keys_out, d_vals_out, n, d_offsets, m, max_len, kt, k, d_ws, ws_bytes,
                          d_merge_costs, true, stream, 0);
}

mps_status mps_batch_autotune(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m, uint64_t n,
                              uint64_t max_len, mps_key_type kt, void* d_ws, size_t ws_bytes, cudaStream_t stream,
                              int* best_k) {
    // every (fan-in, tile) pair: one checked run, then two timed runs
    float best_ms = 0.f;
    TunedCfg best;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return MPS_ERR_CUDA;
    mps_status s = MPS_OK;
    for (int kk : {2, 4, 8}) {
        for (int tile = 0; tile < kTileChoices && s == MPS_OK; tile++) {
            s = batch_dispatch(d_keys_in, nullptr, d_keys_out, nullptr, n, d_offsets, m, max_len, kt, kk, d_ws, ws_bytes,
                               nullptr, true, stream, tile);
            if (s != MPS_OK) break;
            cudaEventRecord(a, stream);
            for (int rep = 0; rep < 2; rep++)
                batch_dispatch(d_keys_in, nullptr, d_keys_out, nullptr, n, d_offsets, m, max_len, kt, kk, d_ws, ws_bytes,
                               nullptr, false, stream, tile);
            cudaEventRecord(b, stream);
            if (cudaEventSynchronize(b) != cudaSuccess) { s = MPS_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (!best.k || ms < best_ms) { best = TunedCfg{kk, tile}; best_ms = ms; }
        }
        if (s != MPS_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != MPS_OK) return s;
    set_tuned_cfg(kt, false, n, m, best);
    if (best_k) *best_k = best.k;
    return MPS_OK;
}

mps_status mps_batch_tuned_config(mps_key_type kt, int has_payload, uint64_t n, uint32_t m, int* k, uint32_t* c_fused,
                                  uint32_t* c_level) {
    if (kt != MPS_U32 && kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    const TunedCfg c = tuned_cfg(kt, has_payload != 0, n, m);
    const MergeGeom g = merge_geom(kt == MPS_U32 ? 4 : 8, has_payload != 0, c.k, c.tile);
    if (k) *k = c.k;
    if (c_fused) *c_fused = g.c_fused;
    if (c_level) *c_level = g.c_level;
    return MPS_OK;
}

mps_status mps_batch_set_config(mps_key_type kt, int has_payload, uint64_t n, uint32_t m, int k, int tile) {
    if (kt != MPS_U32 && kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    if (!fan_in_ok(k)) return MPS_ERR_UNSUPPORTED;
    if (tile < 0 || tile >= kTileChoices) return MPS_ERR_INVALID_ARG;
    set_tuned_cfg(kt, has_payload != 0, n, m, TunedCfg{k, tile});
    return MPS_OK;
}

mps_status mps_batch_graph_create(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m, uint64_t n,
                                  uint64_t max_len, mps_key_type kt, int k, void* d_ws, size_t ws_bytes,
                                  uint64_t* d_merge_costs, cudaStream_t stream, mps_batch_graph** out) {
    if (!out || !stream) return MPS_ERR_INVALID_ARG;
    *out = nullptr;
    // one direct run validates the arguments and sets kernel attributes
    mps_status s = batch_dispatch(d_keys_in, nullptr, d_keys_out, nullptr, n, d_offsets, m, max_len, kt, k, d_ws, ws_bytes,
                                  d_merge_costs, true, stream, 0);
    if (s != MPS_OK) return s;
    mps_batch_graph* g = new mps_batch_graph();
    g->counters = reinterpret_cast<uint64_t*>(d_ws);
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        delete g;
        return MPS_ERR_CUDA;
    }
    s = batch_dispatch(d_keys_in, nullptr, d_keys_out, nullptr, n, d_offsets, m, max_len, kt, k, d_ws, ws_bytes,
                       d_merge_costs, false, stream, 0);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(stream, &graph);
    if (s != MPS_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        delete g;
        return s != MPS_OK ? s : MPS_ERR_CUDA;
    }
    g->graph = graph;
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        return MPS_ERR_CUDA;
    }
    *out = g;
    return MPS_OK;
}

mps_status mps_batch_graph_launch(mps_batch_graph* g, cudaStream_t stream, int check) {
    if (!g || !g->exec) return MPS_ERR_INVALID_ARG;
    if (cudaGraphLaunch(g->exec, stream) != cudaSuccess) return MPS_ERR_CUDA;
    if (check) {
        uint32_t status = 0;
        if (cudaMemcpyAsync(&status, g->counters + kCtrStatus, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
            return MPS_ERR_CUDA;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return MPS_ERR_CUDA;
        if (status) return device_error(status);
    }
    return MPS_OK;
}

mps_status mps_batch_graph_destroy(mps_batch_graph* g) {
    if (!g) return MPS_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return MPS_OK;
}

}  // extern "C"

extern "C" {

void mps_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) {
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_prof.clear();
    g_snap_used = 0;
    g_prof_on = on != 0;
    if (g_prof_on && !g_snap_host) {
        void* h = nullptr;
        if (cudaMallocHost(&h, (size_t)kSnapSlots * kCtrWords * 8) == cudaSuccess) {
            g_snap_host = static_cast<uint64_t*>(h);
            for (int i = 0; i < kSnapSlots; i++) cudaEventCreateWithFlags(&g_snap_ev[i], cudaEventDisableTiming);
        }
    }
}

int mps_profile_read(mps_profile_entry* out, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<mps_profile_entry> agg;
    for (auto& r : g_prof) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        mps_profile_entry* e = nullptr;
        for (auto& x : agg)
            if (!strncmp(x.name, r.name, sizeof(x.name))) e = &x;
        if (!e) {
            agg.push_back(mps_profile_entry{});
            e = &agg.back();
            strncpy(e->name, r.name, sizeof(e->name) - 1);
        }
        e->launches++;
        e->total_ms += ms;
        e->bytes += rec_bytes(r);
    }
    int m = std::min<int>(cap, (int)agg.size());
    for (int i = 0; i < m; i++) out[i] = agg[i];
    return (int)agg.size();
}

mps_status mps_last_stats(mps_stats* out) {
    if (!out) return MPS_ERR_INVALID_ARG;
    const mps_status s = settle_last();
    *out = g_last;
    return s;
}

mps_status mps_sync_status(const void* d_ws, cudaStream_t stream) {
    if (!d_ws) return MPS_ERR_INVALID_ARG;
    uint32_t status = 0;
    const uint64_t* ctr = static_cast<const uint64_t*>(d_ws);  // the counter block opens every workspace
    if (cudaMemcpyAsync(&status, ctr + kCtrStatus, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return MPS_ERR_CUDA;
    return status ? device_error(status) : MPS_OK;
}

const char* mps_status_string(mps_status s) {
    switch (s) {
        case MPS_OK: return "ok";
        case MPS_ERR_INVALID_ARG: return "invalid argument";
        case MPS_ERR_UNSUPPORTED: return "unsupported (k not in {2,4,8} or n >= 2^31)";
        case MPS_ERR_WORKSPACE: return "workspace too small";
        case MPS_ERR_CUDA: return "CUDA runtime error";
        case MPS_ERR_TIMEOUT: return "timed out";
        case MPS_ERR_BUDGET: return "request exceeds the memory budget";
        case MPS_ERR_DEVICE_CHECK: return "device-side check failed";
        case MPS_ERR_NOT_READY: return "not ready";
        case MPS_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

}  // extern "C"
