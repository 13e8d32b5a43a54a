// queue.cu -- request queue with continuous batching (serving).
//
// Clients submit sort requests (device input and output buffers they own).
// A worker thread admits pending requests against a device memory budget --
// a pool the caller hands over at creation -- groups pending requests of
// one kind (uint32 keys, or uint64 keys with uint32 payloads) into a batch,
// gathers their inputs into pool memory laid end to end (one kernel), sorts
// the batch with the batch path (no host synchronisation inside), scatters
// every result to its client's output buffer (one kernel), and records an
// event.  Several batches are in
// flight at once on separate streams, so requests that arrive while others
// run are admitted as soon as pool memory and a stream free up, and their
// work overlaps on the device.  A finished batch releases its pool memory.
// Every wait is bounded; nothing spins on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mps.h"
#include "common.cuh"
#include "pool_alloc.h"

namespace mps {
mps_status batch_dispatch(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out, uint64_t n,
                          const uint64_t* d_off, uint32_t m, uint64_t max_len, mps_key_type kt, int k, void* d_ws,
                          size_t ws_bytes, uint64_t* d_costs, bool sync_at_end, cudaStream_t st, int tile = 0);
}

namespace {

using Clock = std::chrono::steady_clock;

// Per request of a batch: its buffers (keys in, payload in, keys out, payload out).
struct ReqPtrs {
    const void* kin;
    const uint32_t* vin;
    void* kout;
    uint32_t* vout;
};

constexpr uint32_t kSegTile = 4096;  // batch elements per block of the copy kernels

// Moves every request's elements between its own buffers and the batch's
// buffers laid end to end (off[i] = first batch element of request i):
// GATHER copies request inputs into kin/vin, otherwise batch outputs
// kout/vout are scattered to the requests.  A block takes kSegTile batch
// elements, finds the request holding its first one and walks forward.
template <typename K, bool V, bool GATHER>
__global__ void __launch_bounds__(256) k_copy_requests(const ReqPtrs* __restrict__ tab, const uint64_t* __restrict__ off,
                                                       uint32_t m, uint64_t n, K* __restrict__ kin, uint32_t* __restrict__ vin,
                                                       const K* __restrict__ kout, const uint32_t* __restrict__ vout) {
    for (uint64_t x0 = (uint64_t)blockIdx.x * kSegTile; x0 < n; x0 += (uint64_t)gridDim.x * kSegTile) {
        const uint64_t x1 = min(n, x0 + kSegTile);
        uint32_t lo = 0, hi = m;  // last request with off[i] <= x0
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= x0) lo = mid; else hi = mid;
        }
        for (uint32_t i = lo; i < m && off[i] < x1; i++) {
            const uint64_t a = max(off[i], x0), b = min(off[i + 1], x1);
            const ReqPtrs R = tab[i];
            for (uint64_t x = a + threadIdx.x; x < b; x += 256) {
                const uint64_t j = x - off[i];
                if (GATHER) {
                    kin[x] = static_cast<const K*>(R.kin)[j];
                    if (V) vin[x] = R.vin[j];
                } else {
                    static_cast<K*>(R.kout)[j] = kout[x];
                    if (V) R.vout[j] = vout[x];
                }
            }
        }
    }
}

template <typename K, bool V>
void copy_requests(bool gather, const ReqPtrs* tab, const uint64_t* off, uint32_t m, uint64_t n, void* kin, uint32_t* vin,
                   const void* kout, const uint32_t* vout, cudaStream_t st) {
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + kSegTile - 1) / kSegTile, 152 * 8);
    if (gather)
        k_copy_requests<K, V, true><<<grid, 256, 0, st>>>(tab, off, m, n, static_cast<K*>(kin), vin, nullptr, nullptr);
    else
        k_copy_requests<K, V, false><<<grid, 256, 0, st>>>(tab, off, m, n, nullptr, nullptr, static_cast<const K*>(kout),
                                                            vout);
}

void move_requests(bool gather, mps_key_type kt, bool vals, const ReqPtrs* tab, const uint64_t* off, uint32_t m, uint64_t n,
                   void* kin, uint32_t* vin, const void* kout, const uint32_t* vout, cudaStream_t st) {
    if (kt == MPS_U32) {
        if (vals) copy_requests<uint32_t, true>(gather, tab, off, m, n, kin, vin, kout, vout, st);
        else copy_requests<uint32_t, false>(gather, tab, off, m, n, kin, vin, kout, vout, st);
    } else {
        if (vals) copy_requests<uint64_t, true>(gather, tab, off, m, n, kin, vin, kout, vout, st);
        else copy_requests<uint64_t, false>(gather, tab, off, m, n, kin, vin, kout, vout, st);
    }
}

using mps::align_up;
using mps::kPoolAlign;
using mps::PoolAllocator;

struct Ticket {
    mps_request req;
    mps_result res;
    bool done = false;
    Clock::time_point t_submit, t_admit, t_done;
};

struct Batch {
    std::vector<uint64_t> tickets;
    std::vector<std::pair<size_t, size_t>> blocks;  // pool allocations (offset, bytes)
    cudaEvent_t done = nullptr;
    int stream = 0;
};

size_t request_footprint(const mps_request& r) {
    const size_t kb = r.kt == MPS_U32 ? 4 : 8;
    const size_t b = kb + (r.has_payload ? 4 : 0);
    size_t ws = 0;
    mps_batch_workspace_size(r.n, 1, r.kt, r.has_payload, 0, &ws);  // largest over k
    return 2 * align_up(r.n * b) + align_up(ws) + 8 * kPoolAlign;
}

}  // namespace

struct mps_queue {
    mps_queue_config cfg{};
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable cv_done;  // wakes waiters
    std::map<uint64_t, Ticket> tickets;
    std::deque<uint64_t> pending;
    std::vector<Batch> inflight;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;
    std::vector<uint64_t*> h_off;     // pinned offsets staging, one per stream
    // pinned readback, one per stream: the device status word, then at byte 8
    // the merge cost of each request of the stream's batch
    std::vector<uint32_t*> h_status;
    PoolAllocator alloc{0};
    uint64_t next_ticket = 1;
    bool stop = false;
    bool paused = false;
    Clock::time_point t0;
    std::thread worker;
};

namespace {

double ms_since(const Clock::time_point& t0, const Clock::time_point& t) {
    return std::chrono::duration<double, std::milli>(t - t0).count();
}

// Launches one batch of admitted tickets (lock held by the caller).
mps_status launch_batch(mps_queue* q, std::vector<uint64_t>& ids, int sidx, Batch& B) {
    const mps_request& r0 = q->tickets[ids[0]].req;
    const mps_key_type kt = r0.kt;
    const bool vals = r0.has_payload != 0;
    const size_t kb = kt == MPS_U32 ? 4 : 8;
    uint64_t n = 0, max_len = 0;
    for (uint64_t id : ids) {
        n += q->tickets[id].req.n;
        max_len = std::max<uint64_t>(max_len, q->tickets[id].req.n);
    }
    const uint32_t m = (uint32_t)ids.size();
    size_t ws = 0;
    mps_status s = mps_batch_workspace_size(n, m, kt, vals, q->cfg.k ? q->cfg.k : 4, &ws);
    if (s != MPS_OK) return s;
    // offsets (m + 1) and the request pointer table (m) travel in one copy;
    // the per-request merge costs (m) follow them in the same pool block
    const size_t tab_bytes = (size_t)(m + 1) * 8 + (size_t)m * sizeof(ReqPtrs);
    const size_t sizes[6] = {n * kb, n * kb, vals ? n * 4 : 0, vals ? n * 4 : 0, tab_bytes + (size_t)m * 8, ws};
    size_t offs[6];
    for (int i = 0; i < 6; i++) {
        if (!q->alloc.alloc(sizes[i], &offs[i])) {
            for (int j = 0; j < i; j++) q->alloc.release(offs[j], sizes[j]);
            return MPS_ERR_BUDGET;
        }
    }
    for (int i = 0; i < 6; i++) B.blocks.push_back({offs[i], sizes[i]});
    char* pool = static_cast<char*>(q->cfg.d_pool);
    char* kin = pool + offs[0];
    char* kout = pool + offs[1];
    uint32_t* vin = vals ? reinterpret_cast<uint32_t*>(pool + offs[2]) : nullptr;
    uint32_t* vout = vals ? reinterpret_cast<uint32_t*>(pool + offs[3]) : nullptr;
    uint64_t* d_off = reinterpret_cast<uint64_t*>(pool + offs[4]);
    void* d_ws = pool + offs[5];
    cudaStream_t st = q->streams[sidx];
    // the pinned staging buffer of this stream is free: its last copy finished
    // before the stream's previous batch completed
    uint64_t* h_off = q->h_off[sidx];
    ReqPtrs* h_tab = reinterpret_cast<ReqPtrs*>(h_off + (m + 1));
    uint64_t acc = 0;
    for (uint32_t i = 0; i < m; i++) {
        const mps_request& r = q->tickets[ids[i]].req;
        h_off[i] = acc;
        h_tab[i] = ReqPtrs{r.d_keys_in, r.d_vals_in, r.d_keys_out, r.d_vals_out};
        acc += r.n;
    }
    h_off[m] = acc;
    const ReqPtrs* d_tab = reinterpret_cast<const ReqPtrs*>(d_off + (m + 1));
    uint64_t* d_cost = reinterpret_cast<uint64_t*>(pool + offs[4] + tab_bytes);
    cudaMemcpyAsync(d_off, h_off, tab_bytes, cudaMemcpyHostToDevice, st);
    // the stream is idle: no copy into its readback buffer is pending
    uint32_t* h_st = q->h_status[sidx];
    std::memset(h_st, 0, 8 + (size_t)m * 8);
    if (n) {
        move_requests(true, kt, vals, d_tab, d_off, m, n, kin, vin, nullptr, nullptr, st);
        s = mps::batch_dispatch(kin, vin, kout, vout, n, d_off, m, max_len, kt, q->cfg.k ? q->cfg.k : 4, d_ws, ws, d_cost,
                                false, st);
        if (s != MPS_OK) return s;
        // device status word: entry 5 of the workspace's leading 64-bit counter block
        cudaMemcpyAsync(h_st, reinterpret_cast<char*>(d_ws) + 5 * 8, 4, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(reinterpret_cast<char*>(h_st) + 8, d_cost, (size_t)m * 8, cudaMemcpyDeviceToHost, st);
        move_requests(false, kt, vals, d_tab, d_off, m, n, nullptr, nullptr, kout, vout, st);
    }
    if (cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming) != cudaSuccess) return MPS_ERR_CUDA;
    if (cudaEventRecord(B.done, st) != cudaSuccess) return MPS_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return MPS_ERR_CUDA;
    B.tickets = ids;
    B.stream = sidx;
    return MPS_OK;
}

void release_batch(mps_queue* q, Batch& B) {
    for (auto& b : B.blocks) q->alloc.release(b.first, b.second);
    B.blocks.clear();
    if (B.done) cudaEventDestroy(B.done);
    B.done = nullptr;
}

void finish_tickets(mps_queue* q, const std::vector<uint64_t>& ids, mps_status s, uint32_t dev_status = 0,
                    const uint64_t* costs = nullptr) {
    const auto now = Clock::now();
    for (size_t i = 0; i < ids.size(); i++) {
        Ticket& t = q->tickets[ids[i]];
        t.done = true;
        t.t_done = now;
        t.res.status = s;
        t.res.device_status = dev_status;
        t.res.merge_cost = (costs && s == MPS_OK) ? costs[i] : 0;
        t.res.tag = t.req.tag;
        t.res.t_submit_ms = ms_since(q->t0, t.t_submit);
        t.res.t_admit_ms = ms_since(q->t0, t.t_admit);
        t.res.t_done_ms = ms_since(q->t0, now);
    }
}

void worker_main(mps_queue* q) {
    std::unique_lock<std::mutex> lk(q->mu);
    while (true) {
        // 1. retire finished batches
        bool progressed = false;
        for (size_t i = 0; i < q->inflight.size();) {
            Batch& B = q->inflight[i];
            cudaError_t e = cudaEventQuery(B.done);
            if (e == cudaErrorNotReady) { i++; continue; }
            const uint32_t dev = *q->h_status[B.stream];
            mps_status s = MPS_ERR_CUDA;
            if (e == cudaSuccess) s = dev == 0 ? MPS_OK : (dev == mps::kDevSpin ? MPS_ERR_TIMEOUT : MPS_ERR_DEVICE_CHECK);
            // per-request merge costs follow the status word at byte 8
            finish_tickets(q, B.tickets, s, dev, reinterpret_cast<const uint64_t*>(q->h_status[B.stream] + 2));
            q->stream_busy[B.stream] = 0;
            release_batch(q, B);
            q->inflight.erase(q->inflight.begin() + i);
            progressed = true;
        }
        if (progressed) q->cv_done.notify_all();
        if (q->stop && q->inflight.empty()) break;
        // 2. admit and launch: one batch per free stream
        while (!q->stop && !q->paused && !q->pending.empty()) {
            int sidx = -1;
            for (size_t s = 0; s < q->streams.size(); s++)
                if (!q->stream_busy[s]) { sidx = (int)s; break; }
            if (sidx < 0) break;
            const mps_request& head = q->tickets[q->pending.front()].req;
            std::vector<uint64_t> ids;
            size_t need = 0;
            const size_t avail = q->cfg.pool_bytes - q->alloc.used();
            // the oldest request's kind; every pending request of that kind joins, in
            // arrival order, while the batch fits the free budget
            for (auto it = q->pending.begin(); it != q->pending.end() && ids.size() < q->cfg.max_batch; ++it) {
                const mps_request& r = q->tickets[*it].req;
                if (r.kt != head.kt || r.has_payload != head.has_payload) continue;
                size_t f = request_footprint(r);
                if (need + f > avail && !ids.empty()) break;
                ids.push_back(*it);
                need += f;
            }
            if (ids.empty()) break;
            Batch B;
            mps_status s = launch_batch(q, ids, sidx, B);
            if (s == MPS_ERR_BUDGET) {
                release_batch(q, B);
                break;  // wait for memory to free up
            }
            const auto now = Clock::now();
            for (uint64_t id : ids) {
                q->pending.erase(std::find(q->pending.begin(), q->pending.end(), id));
                q->tickets[id].t_admit = now;
            }
            if (s != MPS_OK) {
                // part of the batch may already be queued (the offsets copy,
                // the gather, some sort kernels): let the stream drain before
                // its pool blocks and pinned offsets are reused, and before the
                // callers learn the result and may free their buffers
                cudaStreamSynchronize(q->streams[sidx]);
                release_batch(q, B);
                finish_tickets(q, ids, s);
                q->cv_done.notify_all();
                continue;
            }
            q->stream_busy[sidx] = 1;
            q->inflight.push_back(B);
        }
        // 3. wait for work or completions (bounded; completions are polled)
        if (q->inflight.empty())
            q->cv.wait_for(lk, std::chrono::milliseconds(50));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

mps_status mps_queue_create(const mps_queue_config* cfg, mps_queue** out) {
    if (!cfg || !out || !cfg->d_pool || !cfg->pool_bytes) return MPS_ERR_INVALID_ARG;
    if (cfg->k != 0 && cfg->k != 2 && cfg->k != 4 && cfg->k != 8 && cfg->k != 16) return MPS_ERR_UNSUPPORTED;
    mps_queue* q = new mps_queue();
    q->cfg = *cfg;
    if (!q->cfg.max_inflight) q->cfg.max_inflight = 2;
    if (!q->cfg.max_batch) q->cfg.max_batch = 256;
    if (!q->cfg.timeout_ms) q->cfg.timeout_ms = 10000;
    q->alloc = PoolAllocator(cfg->pool_bytes);
    q->streams.assign(q->cfg.max_inflight, nullptr);
    q->stream_busy.assign(q->cfg.max_inflight, 0);
    q->h_off.assign(q->cfg.max_inflight, nullptr);
    q->h_status.assign(q->cfg.max_inflight, nullptr);
    for (uint32_t i = 0; i < q->cfg.max_inflight; i++) {
        if (cudaStreamCreateWithFlags(&q->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&q->h_off[i], ((size_t)q->cfg.max_batch + 1) * 8 + (size_t)q->cfg.max_batch * sizeof(ReqPtrs)) !=
                cudaSuccess ||
            cudaMallocHost(&q->h_status[i], 8 + (size_t)q->cfg.max_batch * 8) != cudaSuccess) {
            for (uint32_t j = 0; j <= i; j++) {
                if (q->streams[j]) cudaStreamDestroy(q->streams[j]);
                if (q->h_off[j]) cudaFreeHost(q->h_off[j]);
                if (q->h_status[j]) cudaFreeHost(q->h_status[j]);
            }
            delete q;
            return MPS_ERR_CUDA;
        }
    }
    q->t0 = Clock::now();
    q->worker = std::thread(worker_main, q);
    *out = q;
    return MPS_OK;
}

mps_status mps_queue_submit(mps_queue* q, const mps_request* req, uint64_t* ticket) {
    if (!q || !req || !ticket) return MPS_ERR_INVALID_ARG;
    if (req->kt != MPS_U32 && req->kt != MPS_U64) return MPS_ERR_INVALID_ARG;
    if (req->n && (!req->d_keys_in || !req->d_keys_out)) return MPS_ERR_INVALID_ARG;
    if (req->n && req->has_payload && (!req->d_vals_in || !req->d_vals_out)) return MPS_ERR_INVALID_ARG;
    if (req->n >= (1ull << 31)) return MPS_ERR_UNSUPPORTED;
    if (request_footprint(*req) > q->cfg.pool_bytes) return MPS_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(q->mu);
    if (q->stop) return MPS_ERR_CANCELLED;
    const uint64_t id = q->next_ticket++;
    Ticket& t = q->tickets[id];
    t.req = *req;
    t.res = mps_result{};
    t.t_submit = Clock::now();
    q->pending.push_back(id);
    *ticket = id;
    q->cv.notify_one();
    return MPS_OK;
}

mps_status mps_queue_poll(mps_queue* q, uint64_t ticket, mps_result* res) {
    if (!q || !res) return MPS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->tickets.find(ticket);
    if (it == q->tickets.end()) return MPS_ERR_INVALID_ARG;
    if (!it->second.done) return MPS_ERR_NOT_READY;
    *res = it->second.res;
    q->tickets.erase(it);
    return MPS_OK;
}

mps_status mps_queue_wait(mps_queue* q, uint64_t ticket, uint32_t timeout_ms, mps_result* res) {
    if (!q || !res) return MPS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(q->mu);
    auto it = q->tickets.find(ticket);
    if (it == q->tickets.end()) return MPS_ERR_INVALID_ARG;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!q->tickets[ticket].done) {
        if (q->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->tickets[ticket].done)
            return MPS_ERR_TIMEOUT;
    }
    *res = q->tickets[ticket].res;
    q->tickets.erase(ticket);
    return MPS_OK;
}

mps_status mps_queue_pause(mps_queue* q, int paused) {
    if (!q) return MPS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(q->mu);
    q->paused = paused != 0;
    q->cv.notify_one();
    return MPS_OK;
}

mps_status mps_queue_destroy(mps_queue* q) {
    if (!q) return MPS_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
        // pending requests are cancelled; batches in flight drain
        std::vector<uint64_t> cancelled(q->pending.begin(), q->pending.end());
        q->pending.clear();
        finish_tickets(q, cancelled, MPS_ERR_CANCELLED);
        q->cv.notify_one();
        q->cv_done.notify_all();
    }
    if (q->worker.joinable()) q->worker.join();
    for (size_t i = 0; i < q->streams.size(); i++) {
        cudaStreamDestroy(q->streams[i]);
        cudaFreeHost(q->h_off[i]);
        cudaFreeHost(q->h_status[i]);
    }
    delete q;
    return MPS_OK;
}

}  // extern "C"
