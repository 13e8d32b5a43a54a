// kernels.cuh -- workspace view, device records and launcher declarations
// shared by the translation units of the CUDA path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mps {

constexpr int kDetTile = 8192;     // elements per run-detection tile
constexpr int kPackTile = 8192;    // splitter intervals per unit-packing block (64 per thread)
constexpr int kMaskTile = 4096;    // boundaries per mask-scan tile
constexpr int kMaxLevels = 64;     // bound on distinct powers (P <= 32 for n < 2^31)
constexpr int kMinTreeLevels = 8;  // fan-out 32 min-tree over the powers

// Indices into the 64-bit device counter block.
enum : int {
    kCtrR = 0,          // number of runs r
    kCtrLevelBits = 1,  // bit p set if some boundary has power p
    kCtrM = 2,          // merge cost (sum of node sizes)
    kCtrHbmTotal = 3,   // number of nodes executed as level merges
    kCtrFrontier = 4,   // number of fused subtrees (entries of fused_list)
    kCtrStatus = 5,     // device error word (low 32 bits)
    kCtrNodes = 6,      // number of tree nodes
    kCtrUnits = 7,      // work units of the current level
    kCtrHbmCount = 8,   // [64] nodes per power (level merges only)
    kCtrHbmSize = 72,   // [64] elements per power (level merges only)
    kCtrHbmFill = 136,  // [64] fill counters for bucketing
    kCtrSplits = 201,   // splitters of the current level
    kCtrIntervals = 202,  // splitter intervals of the current level (packed into units)
    kCtrMaxRun = 203,   // longest run (elements)
    kCtrMaxLen = 204,   // longest array of a batch (elements)
    kCtrCand = 206,     // node-pass candidates listed by the mask pass
    kCtrMrGood = 207,   // minimum run length: good intervals (natural runs of >= m-1 interior flags)
    kCtrTailCount = 208,  // final-collapse variant: boundaries left on the run stack after the last run
    kCtrTailShift = 209,  // final-collapse variant: number of final-collapse nodes (added to every other power)
    kCtrFusedNext = 210,  // next fused tile to take (dynamic scheduling of k_fused)
    kCtrWords = 256
};

// Largest fan-in k (and node degree) the kernels take: k in {2, 4, 8, 16}.
constexpr int kMaxFanIn = 16;
inline bool fan_in_ok(int k) { return k == 2 || k == 4 || k == 8 || k == 16; }
// bytes of one level-merge work-unit descriptor
constexpr size_t kUnitDescBytes = 192;

// A node executed by the level-merge kernels (more than T_max elements).
// Children c = 0..d-1 cover runs [b[c], b[c+1]); b[0] and b[d] are the node's
// delimiting boundaries (nearest boundaries of smaller power).
struct __align__(16) LevelNode {
    uint32_t sL, sR;          // element range of the node
    uint32_t unit_off;        // first work unit of this node (per level)
    uint32_t nunits;          // number of work units
    uint32_t b[kMaxFanIn + 1];  // child boundaries (run indices)
    uint8_t power, depth, degree, pad;
    uint32_t split_off;       // first splitter of this node (per level)
    uint32_t nsplit;          // number of splitters
};
static_assert(sizeof(LevelNode) == 96, "LevelNode layout");

struct WsView {
    uint64_t n;                    // keys being sorted (all arrays of a batch)
    uint64_t* counters;
    uint64_t* det_state;           // run detection: tile summaries, tile prefixes, comparison bits
    uint32_t* run_starts;
    uint8_t* run_desc;
    uint8_t* lv[kMinTreeLevels];   // lv[0] = powers[0..r] (+ padding)
    uint32_t lv_len[kMinTreeLevels];
    int nlv;
    uint8_t* powers;               // == lv[0]
    uint8_t* node_info;            // [b] for boundary j = b + 1: depth | needs_query << 6 | is_start << 7
    unsigned long long* mt_f;      // mask-scan tile aggregates
    unsigned long long* mt_g;
    unsigned long long* mt_fpre;
    unsigned long long* mt_gsuf;
    uint4* fused_list;             // fused subtrees: {first run, end run, depth, 0}
    uint32_t fused_cap;
    uint32_t* level_off;           // [64] first bucket entry of each power
    LevelNode* nodes_raw;
    LevelNode* nodes_lvl;
    uint32_t nodes_cap;
    uint32_t* unit_node;
    uint32_t* split_tab;
    void* unit_desc;               // 128-byte work-unit descriptors of the current level
    uint32_t* unit_first;          // first splitter interval of each packed work unit
    uint32_t* pack_tiles;          // per-tile counts / offsets of the packing scan
    uint32_t* ivl_size;            // [unit_cap + 64] interval sizes, bit 31 = first interval of its node
    uint32_t unit_cap;
    uint32_t* canon_idx;           // dump: canonical index of each node start; before that, the
                                   // node pass's candidate list (boundary indices)
    uint32_t cand_cap;             // entries of canon_idx
    uint32_t* hist;                // dump: per-tile power histograms
    uint32_t* tail_list;           // final-collapse variant: boundaries left on the run stack (kTailCap)
    void* keys_tmp;
    uint32_t* vals_tmp;
    // batch of arrays laid end to end (nullptr for a single array)
    const uint64_t* batch_off;     // [m+1] array starts, batch_off[m] = n
    uint32_t batch_m;
    uint64_t batch_max_len;        // caller's bound on the longest array (0: none)
    uint64_t* batch_cost;          // [m] merge cost per array, or nullptr
    uint2* batch_prm;              // [2m] per-array power parameters
};

// Buffers of the minimum-run-length partition (Sec. 5, "Minimal run length").
// A good interval j is the set [gs[j], ge[j]) of positions from which the
// natural run is at least m long; all of them end their run at v[j].  Node 0
// is position 0, node j + 1 the position v[j]; every node knows the node its
// run progression reaches next (succ), the start of the natural run that ends
// the progression (hit, n if none), and how many runs it contributes (cnt).
struct MinRunView {
    uint32_t m;            // minimum run length, 2..32
    uint32_t cap;          // capacity of the good-interval and node arrays
    uint32_t* gs;
    uint32_t* ge;
    uint32_t* gv;
    uint32_t* succ;
    uint32_t* hit;
    uint32_t* cnt;
    uint32_t* off;         // run index of each node's first run (marked nodes)
    uint32_t* mark;        // node on the chain from position 0
    uint32_t* jmp0;        // pointer-jumping buffers
    uint32_t* jmp1;
    uint32_t* tiles;       // per-tile counts and offsets of the two scans
    uint32_t tiles_cap;
    uint8_t* desc_nat;     // direction of each run's natural part (tree output)
};

// Sizes of the merge stages for one key/payload type.
struct MergeGeom {
    uint32_t c_fused;   // elements of shared memory per fused tile
    uint32_t tmax;      // largest fused subtree (== c_fused)
    uint32_t c_level;   // elements per level-merge unit
    uint32_t ts;        // splitter spacing per child (c_level / k)
    int k;              // fan-in
    uint32_t level_grid;  // blocks of the persistent level merge
    uint32_t fused_grid;  // blocks of the persistent fused-subtree kernel
};

// Tile choices for the merge stages of one key/payload type: 0 is the
// default; 1 and 2 trade the fused tile's size against the blocks that share
// an SM (items per thread = c_fused / 256).
constexpr int kTileChoices = 3;
MergeGeom merge_geom(int key_bytes, bool vals, int k, int tile = 0);

// Number of kernels launched by this thread since the counter was last reset.
extern thread_local uint64_t g_launches;

// runs.cu
template <typename K> void launch_detect(const K* keys, uint64_t n, const WsView& ws, cudaStream_t st);
void launch_powers(uint64_t n, uint32_t r, int k, const WsView& ws, cudaStream_t st);

// tail.cu: a final collapse other than the power rule (policy 1: Alg. 2's
// last loop as printed, pop k-1 runs per merge; policy 2: the appendix's
// merge_down) by relabelling ws.powers so that the power rule builds that
// tree.  orig_powers, if given, receives the powers before relabelling (r+1
// entries).  Sets ctr[kCtrTailShift].
constexpr uint32_t kTailCap = 512;
void launch_tail(uint32_t r_bound, int k, int policy, uint8_t* orig_powers, const WsView& ws, cudaStream_t st);

// tree.cu
void launch_mintree(uint32_t r, const WsView& ws, cudaStream_t st);
void launch_masks(uint32_t r, bool dump_leaf, uint8_t* leaf_depth, uint64_t n, int k, uint32_t tmax, const WsView& ws,
                  cudaStream_t st);
// vmax: largest power for which level merges are queued (a larger node at a
// higher power is reported as device status kDevLevelBound)
void launch_node_pass(uint32_t r, int k, uint32_t tmax, uint32_t vmax, const WsView& ws, cudaStream_t st);
void launch_bucket(uint32_t total_bound, const WsView& ws, cudaStream_t st);
// Canonical tree of the last sort (r read on the device, r <= r_bound).
void launch_tree_dump(uint32_t r_bound, int k, const WsView& ws, uint32_t* node_first, void* nodes, cudaStream_t st);
// Run starts, directions (from desc_src), powers and counts {r, nodes,
// levels, M} of the last sort copied to the caller's tree arrays (any may be null).
void launch_tree_arrays(uint32_t r_bound, const WsView& ws, const uint8_t* desc_src, uint32_t* run_starts, uint8_t* run_desc,
                        uint8_t* powers, uint8_t* leaf_depth, uint64_t* counts, cudaStream_t st);

// merge.cu
template <typename K, bool V>
void launch_fused(const K* leaf_keys, const uint32_t* leaf_vals, K* out, uint32_t* vout, uint64_t nfused,
                  const MergeGeom& g, const WsView& ws, cudaStream_t st);
// One power level p of the level merges.  nn_bound / elems_bound bound the
// level's node and element counts (exact values are read on the device).
template <typename K>
void launch_level_plan(int p, uint32_t nn_bound, uint64_t elems_bound, int k, const K* leaf_keys, K* out,
                       const MergeGeom& g, const WsView& ws, cudaStream_t st);
template <typename K, bool V>
void launch_level_merge(uint32_t nn_bound, uint64_t elems_bound, const K* leaf_keys, const uint32_t* leaf_vals, K* out,
                        uint32_t* vout, const MergeGeom& g, const WsView& ws, cudaStream_t st);
// minrun.cu: replaces the natural run partition in ws (run_starts, run
// direction, r) by the minimum-run-length partition; `copy` holds a copy of
// the keys (and payloads) into which every run of at most m elements is
// sorted stably.  ws.run_desc then flags only the natural runs longer than m
// that are strictly descending (read backwards by the merges).
template <typename K, bool V>
void launch_min_run(const K* keys, K* copy, uint32_t* vcopy, uint64_t n, const MinRunView& mr, const WsView& ws,
                    cudaStream_t st);

template <typename K, bool V>
void launch_copy_single_run(const K* in, const uint32_t* vin, K* out, uint32_t* vout, uint64_t n,
                            const WsView& ws, cudaStream_t st);
// Batches: arrays that consist of a single run are copied (reversed if
// strictly descending) straight to the output.
template <typename K, bool V>
void launch_copy_lone_runs(const K* in, const uint32_t* vin, K* out, uint32_t* vout, uint32_t r_bound,
                           const WsView& ws, cudaStream_t st);

}  // namespace mps
