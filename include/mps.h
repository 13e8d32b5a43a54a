/*
 * mps.h -- C ABI of the GB300-native Multiway Powersort library (libmps.so).
 *
 * The library sorts device arrays with Multiway Powersort (Cawley Gelling,
 * Nebel, Smith, Wild, arXiv 2209.06909): it detects the input's natural runs
 * (maximal weakly increasing or strictly decreasing segments, the latter
 * reversed; Sec. 2), computes every run boundary's k-way power (Def. 3.1),
 * builds the merge tree those powers define (Alg. 1) and executes it level by
 * level as stable k-way merges (Sec. 2.2, Sec. 4).  Every step runs in CUDA
 * kernels written for sm_103a; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers owned by the caller; the library
 *     never allocates or frees device memory on these paths.  Host pointers
 *     are named h_*.
 *   - Calls are enqueued on the given CUDA stream.  mps_sort_keys,
 *     mps_sort_pairs, mps_merge_tree, mps_sort_keys_noalloc and
 *     mps_sort_records return as soon as their kernels are queued: every
 *     launch is sized by bounds from n and reads the actual counts (runs,
 *     nodes, work units) from the workspace, so no host thread waits for the
 *     device.  Outputs are complete in stream order (synchronise the stream,
 *     or queue later work on it, before reading them).  A device-side check
 *     failure is recorded in the workspace's status word; mps_sync_status or
 *     mps_last_stats (both synchronise the stream) report it.
 *   - Key types: MPS_U32 (uint32_t) or MPS_U64 (uint64_t), compared as
 *     unsigned integers; every value, including the type's maximum, is a
 *     legal key (no sentinel is reserved; cf. Sec. 4 "Sentinel values").
 *   - Fan-in k must be 2, 4, 8 or 16 (Sec. 3's k-way powers for k a power of
 *     two; Sec. 6 leaves k > 4 open).  n must be below 2^32 (below 2^31 with a
 *     minimum run length, and for a queued request).
 *   - For a single array, d_keys_out may equal (or overlap) d_keys_in, and
 *     d_vals_out d_vals_in: the sort then reads a copy of the input that it
 *     makes in the workspace (mps_workspace_size includes room for it).  Keys
 *     and payloads must not overlap each other.  Batch outputs must not
 *     overlap their inputs.
 *   - A workspace serves one call at a time.  Two calls whose kernels may run
 *     at the same time (queued on different streams with no event or
 *     synchronisation between them) need different workspaces: sharing one
 *     mixes the two sorts' counters and tables, and kernels that index with
 *     them can then read or write out of range.
 *   - Errors are returned as mps_status; a device-side invariant violation
 *     (which would indicate a library bug) is reported as MPS_ERR_DEVICE_CHECK.
 */
#ifndef MPS_H
#define MPS_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPS_OK = 0,
    MPS_ERR_INVALID_ARG = 1,  /* null pointer, overlap, bad key type           */
    MPS_ERR_UNSUPPORTED = 2,  /* k not in {2,4,8,16}, n >= 2^32 (see above)     */
    MPS_ERR_WORKSPACE = 3,    /* workspace smaller than mps_workspace_size      */
    MPS_ERR_CUDA = 4,         /* a CUDA runtime call failed                     */
    MPS_ERR_TIMEOUT = 5,      /* a bounded wait ran out (queue / device spin)   */
    MPS_ERR_BUDGET = 6,       /* request larger than the serving budget         */
    MPS_ERR_DEVICE_CHECK = 7, /* a device-side invariant check failed           */
    MPS_ERR_NOT_READY = 8,    /* queue: ticket still in flight                  */
    MPS_ERR_CANCELLED = 9     /* queue: request cancelled by destroy            */
} mps_status;

typedef enum { MPS_U32 = 0, MPS_U64 = 1 } mps_key_type;

/* One node of the canonical merge-tree encoding (16 bytes).  A node covers
 * the runs [first_run, end_run); its d-1 run boundaries all carry the power
 * `power` (Sec. 2.2: each merge-tree node of degree d owns d-1 boundaries).
 * The table is sorted by (power, first_run); `parent` indexes that table and
 * is 0xFFFFFFFF at the root. */
typedef struct {
    uint32_t first_run;
    uint32_t end_run;
    uint8_t power;
    uint8_t degree;
    uint16_t pad;
    uint32_t parent;
} mps_node;

/* Optional tree outputs (all device pointers, caller-allocated, sized for the
 * worst case of n runs).  Any member may be NULL to skip it.
 *   run_starts[n+1] : s_0 = 0 < s_1 < ... < s_r = n (Sec. 2, runs R_0..R_{r-1})
 *   run_desc[n]     : 1 if run i was strictly decreasing (and got reversed)
 *   powers[n+1]     : powers[i] = P_i of boundary B_i (1 <= i < r), Def. 3.1;
 *                     powers[0] = powers[r] = 0
 *   node_first[n]   : smallest boundary index of the node owning B_i
 *                     (node_first[0] = 0)
 *   nodes[n]        : canonical node table (see mps_node)
 *   leaf_depth[n]   : d_i, the depth of run i in the tree (Sec. 2.2)
 *   counts[4]       : {r, number of nodes, number of distinct powers,
 *                      merge cost M = sum_i d_i L_i} (Sec. 2.2)            */
typedef struct {
    uint32_t* run_starts;
    uint8_t* run_desc;
    uint8_t* powers;
    uint32_t* node_first;
    mps_node* nodes;
    uint8_t* leaf_depth;
    uint64_t* counts;
} mps_tree;

/* Bytes of device workspace needed to sort n keys of type kt (with a uint32
 * payload if has_payload) with fan-in k.  The same size serves
 * mps_merge_tree.  Returns MPS_ERR_INVALID_ARG if bytes is NULL. */
mps_status mps_workspace_size(uint64_t n, mps_key_type kt, int has_payload, int k, size_t* bytes);

/* Multiway Powersort of n keys (Alg. 2's merge policy via the tree of Alg. 1).
 *   d_keys_in  : n keys, read only.
 *   d_keys_out : n keys, receives the sorted keys.
 *   d_ws       : workspace of at least mps_workspace_size(n, kt, 0, k) bytes.
 *   opt_tree   : NULL, or device arrays that receive the run structure,
 *                powers and canonical tree (slower: builds the full table). */
mps_status mps_sort_keys(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k,
                         void* d_ws, size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream);

/* Stable key-value sort: every uint32 payload moves with its key, and equal
 * keys keep their input order (runs are weakly increasing or strictly
 * decreasing, so reversal never reorders equal keys; merges prefer the
 * leftmost run on ties -- Sec. 2, Sec. 4 "Tournament tree").
 * Workspace: mps_workspace_size(n, kt, 1, k). */
mps_status mps_sort_pairs(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out,
                          uint32_t* d_vals_out, uint64_t n, mps_key_type kt, int k,
                          void* d_ws, size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream);

/* Multiway Powersort with a minimum run length (Sec. 5, "Minimal run
 * length": the paper's experiments extend runs to 24 elements).  Runs are
 * found greedily from the left as in mps_sort_keys, except that a natural run
 * shorter than min_run_len is extended to min_run_len elements (or to the end
 * of the array) and sorted stably; the next run is searched from the end of
 * the extended one.  Powers, tree and merges then follow Def. 3.1 and Alg. 1
 * on these runs.  min_run_len = 1 is mps_sort_keys; 2..32 are supported
 * (MPS_ERR_UNSUPPORTED otherwise).  opt_tree->run_desc flags the runs whose
 * natural part was strictly decreasing.  Workspace:
 * mps_workspace_size_minrun(n, kt, has_payload, k, min_run_len). */
mps_status mps_workspace_size_minrun(uint64_t n, mps_key_type kt, int has_payload, int k, uint32_t min_run_len,
                                     size_t* bytes);
mps_status mps_sort_keys_minrun(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k,
                                uint32_t min_run_len, void* d_ws, size_t ws_bytes, const mps_tree* opt_tree,
                                cudaStream_t stream);
/* Stable key-value form of mps_sort_keys_minrun. */
mps_status mps_sort_pairs_minrun(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out,
                                 uint32_t* d_vals_out, uint64_t n, mps_key_type kt, int k, uint32_t min_run_len,
                                 void* d_ws, size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream);

/* Multiway Powersort whose run stack is emptied after the last run by a
 * policy other than the power rule (Alg. 2's main loop is unchanged):
 *   tail_policy 0: the power rule against a final power 0 -- Alg. 1's tree,
 *                  exactly mps_sort_keys;
 *   tail_policy 1: Alg. 2's last loop as printed: pop up to k-1 stack entries
 *                  per merge with the current run;
 *   tail_policy 2: the appendix's merge_down (written for k = 4, here for any
 *                  k): first merge the top (entries mod (k-1)) entries with the
 *                  current run, then k-1 entries per merge.
 * For k = 2 the three build the same tree.  The sorted keys are those of
 * mps_sort_keys; the tree (opt_tree: node table, node_first, leaf depths,
 * counts with the merge cost M of Sec. 2.2) is the policy's.  opt_tree->powers
 * receives the powers of Def. 3.1; the node table's power field holds the
 * labels the tree was built from: each final-collapse node is numbered from
 * the root (1, 2, ...) and every other power is raised by the number of
 * final-collapse nodes.  Workspace: mps_workspace_size(n, kt, 0, k).  Device
 * status 20 if the relabelled powers would exceed 32 (possible above n = 2^30
 * at k = 4).
 * tail_policy outside 0..2: MPS_ERR_INVALID_ARG. */
mps_status mps_sort_keys_tail(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k, int tail_policy,
                              void* d_ws, size_t ws_bytes, const mps_tree* opt_tree, cudaStream_t stream);

/* Records (Sec. 5, "records" experiment: a long key and a pointer, 16 bytes):
 * stable sort of n keys each carrying a 64-bit payload.  The keys are sorted
 * with their input indices as uint32 payloads (as mps_sort_pairs), and every
 * payload is then moved once through that stable permutation:
 * d_vals_out[i] = d_vals_in[perm[i]].  d_vals_in and d_vals_out must not
 * overlap.  Workspace: mps_records_workspace_size(n, kt, k) bytes (the pairs
 * workspace plus 8 bytes per key).  Returns once its kernels are queued. */
mps_status mps_records_workspace_size(uint64_t n, mps_key_type kt, int k, size_t* bytes);
mps_status mps_sort_records(const void* d_keys_in, const uint64_t* d_vals_in, void* d_keys_out,
                            uint64_t* d_vals_out, uint64_t n, mps_key_type kt, int k, void* d_ws,
                            size_t ws_bytes, cudaStream_t stream);

/* Run structure, powers and canonical merge tree of d_keys without moving
 * any key (the keys are not modified).  `out` must be non-NULL. */
mps_status mps_merge_tree(const void* d_keys, uint64_t n, mps_key_type kt, int k, const mps_tree* out,
                          void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* End-to-end form of mps_sort_keys from host memory: copies h_keys_in to
 * d_keys_in, sorts into d_keys_out and copies the result to h_keys_out, all on
 * `stream` (pinned host buffers give asynchronous copies).  Returns after the
 * result has reached h_keys_out. */
mps_status mps_sort_keys_host(const void* h_keys_in, void* h_keys_out, uint64_t n, mps_key_type kt, int k,
                              void* d_keys_in, void* d_keys_out, void* d_ws, size_t ws_bytes,
                              cudaStream_t stream);

/* The same three steps queued on `stream` without waiting: the call returns
 * once the input copy, the sort's kernels and the output copy are enqueued,
 * and h_keys_out holds the result when `stream` reaches that point.  With
 * pinned host buffers the copies run on the copy engines, so a caller that
 * sorts a sequence of arrays on two or more streams (each with its own device
 * buffers and workspace) overlaps one array's copies with another's sort.
 * The host buffers, device buffers and workspace must stay untouched until
 * the stream has passed the call.  The sort's argument checks (key type, k,
 * n, workspace size and alignment) come first, so a rejected call queues
 * nothing.  Returns MPS_ERR_CUDA if a copy cannot be queued; other errors as
 * mps_sort_keys (device-side failures are read with mps_sync_status). */
mps_status mps_sort_keys_host_async(const void* h_keys_in, void* h_keys_out, uint64_t n, mps_key_type kt, int k,
                                    void* d_keys_in, void* d_keys_out, void* d_ws, size_t ws_bytes,
                                    cudaStream_t stream);

/* ---------------------------------------------------------------- batches
 * A batch is m independent arrays laid end to end in one key buffer:
 * array a occupies [d_offsets[a], d_offsets[a+1]) with d_offsets[0] = 0 and
 * d_offsets[m] = n (device memory, non-decreasing; empty arrays allowed).
 * Every array is sorted on its own with its own runs, powers (Def. 3.1 with
 * the array's length) and merge tree; one pass of each kernel covers all
 * arrays, and the launch sequence makes no host synchronisation, so it can be
 * captured in a CUDA graph (see mps_batch_graph_*).
 *   max_len : an upper bound on the longest array (sizes the level loop);
 *             0 means n.  An array longer than max_len is detected on the
 *             device and reported as MPS_ERR_DEVICE_CHECK (status 16).
 *   k       : 2, 4, 8 or 16 with the default tiles, or 0 for the configuration
 *             (fan-in and tile sizes) chosen by mps_batch_autotune or set by
 *             mps_batch_set_config for this key type and mean array size
 *             (k = 4, default tiles until then).
 * n must be below 2^32.  Workspace: mps_batch_workspace_size(n, m, kt,
 * has_payload, k); k = 0 asks for the largest over every configuration.
 *   d_merge_costs : NULL, or device memory for m uint64 values that receives
 *             each array's merge cost M = sum_i depth(run i) * L_i (Sec. 2.2)
 *             in its own tree, the same value as sorting the array alone (0
 *             for arrays of at most one run).  Written in stream order; a
 *             graph (mps_batch_graph_*) rewrites it at every replay.
 * mps_sort_batch and mps_sort_batch_pairs synchronise the stream once at the
 * end to report device-side check failures. */
mps_status mps_batch_workspace_size(uint64_t n, uint32_t m, mps_key_type kt, int has_payload, int k, size_t* bytes);

mps_status mps_sort_batch(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m, uint64_t n,
                          uint64_t max_len, mps_key_type kt, int k, void* d_ws, size_t ws_bytes,
                          uint64_t* d_merge_costs, cudaStream_t stream);

/* Stable key-value form of mps_sort_batch (uint32 payload per key). */
mps_status mps_sort_batch_pairs(const void* d_keys_in, const uint32_t* d_vals_in, void* d_keys_out,
                                uint32_t* d_vals_out, const uint64_t* d_offsets, uint32_t m, uint64_t n,
                                uint64_t max_len, mps_key_type kt, int k, void* d_ws, size_t ws_bytes,
                                uint64_t* d_merge_costs, cudaStream_t stream);

/* Times the batch (keys only; the output buffer is overwritten) for every
 * fan-in k in {2, 4, 8} and every tile choice, and records the fastest pair
 * for this key type and mean array size (log2 of n / m); later calls with
 * k = 0 use it.  *best_k receives the fan-in; mps_batch_tuned_config reports
 * the tile sizes.  A tile choice sets the fused-subtree tile (elements merged
 * in one block's shared memory; items per thread = tile / 256) and the
 * level-merge work unit: choice 0 is the default (4096 and 9216 elements for
 * uint32 keys); 1 and 2 are other sizes (for uint32 keys a larger fused tile
 * with fewer blocks per SM, and smaller tiles).  The
 * workspace must be sized with k = 0. */
mps_status mps_batch_autotune(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m,
                              uint64_t n, uint64_t max_len, mps_key_type kt, void* d_ws, size_t ws_bytes,
                              cudaStream_t stream, int* best_k);

/* The configuration that k = 0 selects for batches of this key type,
 * payload flag and mean array size n / m: fan-in, fused-subtree tile and
 * level-merge unit (elements). */
mps_status mps_batch_tuned_config(mps_key_type kt, int has_payload, uint64_t n, uint32_t m, int* k, uint32_t* c_fused,
                                  uint32_t* c_level);
/* Sets that configuration by hand: k in {2, 4, 8, 16}, tile in 0..2 (0: the
 * default tiles; 1, 2: the other choices of mps_batch_autotune). */
mps_status mps_batch_set_config(mps_key_type kt, int has_payload, uint64_t n, uint32_t m, int k, int tile);

/* A batch sort captured once into a CUDA graph for the given buffers (the
 * graph replays the whole kernel sequence; the buffers must stay valid).
 * create runs the batch once directly, then captures it on `stream` (which
 * must not be the legacy default stream).  launch enqueues one replay; with
 * check != 0 it also synchronises and reports device-side check failures. */
typedef struct mps_batch_graph mps_batch_graph;
mps_status mps_batch_graph_create(const void* d_keys_in, void* d_keys_out, const uint64_t* d_offsets, uint32_t m,
                                  uint64_t n, uint64_t max_len, mps_key_type kt, int k, void* d_ws, size_t ws_bytes,
                                  uint64_t* d_merge_costs, cudaStream_t stream, mps_batch_graph** out);
mps_status mps_batch_graph_launch(mps_batch_graph* g, cudaStream_t stream, int check);
mps_status mps_batch_graph_destroy(mps_batch_graph* g);

/* ---------------------------------------------------------------- serving
 * A request queue with continuous batching.  Clients submit sort requests on
 * device buffers they own (inputs must stay unchanged and outputs untouched
 * until the request completes).  A worker thread admits pending requests
 * against a device memory budget -- the pool the caller hands over at
 * creation -- gathers the pending requests of the oldest request's kind into
 * a batch, stages their inputs in the pool, sorts the batch (mps_sort_batch's
 * kernels, no host synchronisation), and copies each result to its client's
 * output.
 * Up to max_inflight batches run at once on separate streams, so requests
 * that arrive while others are on the GPU are admitted as pool memory and a
 * stream free up, and their work overlaps on the device.  Each result is
 * exactly the sort the request would get alone. */
typedef struct {
    void* d_pool;           /* device memory owned by the caller, used as the budget */
    size_t pool_bytes;      /* admission budget in bytes */
    uint32_t max_inflight;  /* batches (streams) in flight, 0 -> 2 */
    uint32_t max_batch;     /* requests per batch, 0 -> 256 */
    uint32_t timeout_ms;    /* reserved for bounded waits, 0 -> 10000 */
    int k;                  /* fan-in 2, 4, 8 or 16; 0 -> 4 */
} mps_queue_config;

typedef struct {
    mps_key_type kt;        /* MPS_U32 or MPS_U64 keys */
    int has_payload;        /* 1: uint32 payload per key (stable) */
    uint64_t n;
    const void* d_keys_in;
    const uint32_t* d_vals_in;
    void* d_keys_out;
    uint32_t* d_vals_out;
    uint64_t tag;           /* returned in the result */
} mps_request;

typedef struct {
    mps_status status;      /* MPS_OK, MPS_ERR_CANCELLED, MPS_ERR_DEVICE_CHECK, ... */
    uint32_t device_status; /* device-side check code when status is MPS_ERR_DEVICE_CHECK */
    uint64_t tag;
    uint64_t merge_cost;    /* M of Sec. 2.2 for this request's array (0 unless status is MPS_OK) */
    double t_submit_ms, t_admit_ms, t_done_ms;  /* milliseconds since the queue was created */
} mps_result;

typedef struct mps_queue mps_queue;

/* Starts the worker thread and its streams.  MPS_ERR_INVALID_ARG if the pool
 * is missing; the pool stays the caller's and must outlive the queue. */
mps_status mps_queue_create(const mps_queue_config* cfg, mps_queue** q);
/* Enqueues a request; *ticket identifies it.  MPS_ERR_BUDGET if the request
 * alone cannot fit the budget, MPS_ERR_INVALID_ARG for missing buffers. */
mps_status mps_queue_submit(mps_queue* q, const mps_request* req, uint64_t* ticket);
/* MPS_ERR_NOT_READY while the request is pending or in flight; otherwise
 * fills *res and forgets the ticket. */
mps_status mps_queue_poll(mps_queue* q, uint64_t ticket, mps_result* res);
/* Waits at most timeout_ms for the request (MPS_ERR_TIMEOUT otherwise). */
mps_status mps_queue_wait(mps_queue* q, uint64_t ticket, uint32_t timeout_ms, mps_result* res);
/* Holds (1) or resumes (0) admission of new batches; batches in flight run on. */
mps_status mps_queue_pause(mps_queue* q, int paused);
/* Cancels pending requests (status MPS_ERR_CANCELLED), drains batches in
 * flight, stops the worker. */
mps_status mps_queue_destroy(mps_queue* q);

/* Sort without any device allocation by the caller or the library (no
 * counterpart in the paper: this is a deployment convenience).  Meant for
 * callers that cannot call cudaMalloc when they need a sort -- code running
 * inside a memory pool it does not own, plugin hosts that forbid device
 * allocations after start-up, or latency-critical paths where an allocation
 * and its implicit synchronisation are not allowed.  The caller passes only
 * its input and output arrays; the workspace is a 32 MiB scratch array
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.
 *   n      : at most 2^20 keys (uint32 or uint64, any k in {2,4,8,16});
 *            larger n returns MPS_ERR_WORKSPACE without touching the GPU.
 *   Other arguments and outputs are those of mps_sort_keys (no tree output).
 * Like mps_sort_keys, the call returns once its kernels are queued; the host
 * does not wait for the device.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for later
 * calls; make that first call before any stream capture.  cudaDeviceReset
 * invalidates the kept address: after a reset, do not call this function
 * again in the same process.  All calls on a device share the one scratch
 * array, which keeps the previous call's contents (the sort clears what it
 * needs zeroed), so calls that overlap on the GPU -- e.g. from two host
 * threads or on two streams at once -- race and must be serialised. */
mps_status mps_sort_keys_noalloc(const void* d_keys_in, void* d_keys_out, uint64_t n, mps_key_type kt, int k,
                                 cudaStream_t stream);

/* Per-kernel timing with CUDA events recorded on the launching stream.
 * mps_profile_enable(1) clears and starts recording; mps_profile_read fills
 * up to `cap` entries (kernel name, launches, total milliseconds) after
 * synchronising the recorded events, and returns the number of entries. */
typedef struct {
    char name[48];
    uint64_t launches;
    double total_ms;
    double bytes;      /* algorithmic bytes moved by those launches */
} mps_profile_entry;

void mps_profile_enable(int on);
int mps_profile_read(mps_profile_entry* out, int cap);

/* Synchronises `stream` and returns the device-side status of the last sort
 * or batch that used the workspace d_ws: MPS_OK, MPS_ERR_DEVICE_CHECK (an
 * invariant check failed; mps_last_stats gives the code) or MPS_ERR_TIMEOUT (a
 * bounded device wait ran out).  No counterpart in the paper. */
mps_status mps_sync_status(const void* d_ws, cudaStream_t stream);

/* Statistics of the most recent sort on this host thread (host memory).  For
 * a single-array sort the statistics live in its workspace on the device: this
 * call synchronises that sort's stream and reads them back, so that workspace
 * must still be allocated, and not handed to another call, until then. */
typedef struct {
    uint64_t n, r, merge_cost, frontier_nodes, hbm_nodes;
    uint32_t num_levels, hbm_levels;
    uint64_t bytes_fused, bytes_levels; /* algorithmic bytes of the merge kernels */
    uint64_t launches;                  /* CUDA kernels launched by the call */
    uint32_t device_status;             /* device-side check code (0 = none): 1 node degree > k,
                                           2 capacity, 3 tile overflow, 11-15 work-unit / fused /
                                           lone-run ranges, 16 array longer than max_len, 17 a
                                           bounded wait ran out (returned as MPS_ERR_TIMEOUT),
                                           18 a splitter ranked outside its node (unsorted child),
                                           19 a node above the fused-tile size at a power beyond
                                           the levels queued for it, 20 final-collapse relabelling
                                           out of range (mps_sort_keys_tail) */
    uint32_t pad;
} mps_stats;

mps_status mps_last_stats(mps_stats* out);

const char* mps_status_string(mps_status s);

#ifdef __cplusplus
}
#endif

#endif /* MPS_H */
