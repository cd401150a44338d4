// rs_server.cu -- a sort server: requests arrive at any time from any host
// thread; a dispatcher thread admits them under a device-memory budget, packs
// waiting small radix requests with the same key type into one segmented sort
// (continuous batching), runs large requests on their own, and keeps several
// launches in flight on separate streams so their work overlaps on the GPU.
// Completion is observed through CUDA events.  Every request's result is the
// same as sorting it alone with rs_sort_* / bs_sort_* (each segment of a
// batch is sorted independently, stably).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rs_segmented.h"

namespace rs {

size_t segmented_workspace_bytes(int key_bytes, bool vals, size_t n_total, size_t nseg, int key_bits);
size_t bucket_workspace_bytes(int key_bytes, bool vals, size_t n, size_t nb);
size_t seg_bucket_workspace_bytes(int key_bytes, bool vals, size_t n_total, size_t nseg, size_t keys_per_bucket);

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over the caller's device pool (256-byte granules).
class PoolAllocator {
  public:
    void init(void* base, size_t bytes) {
        base_ = static_cast<unsigned char*>(base);
        free_.clear();
        if (bytes >= 256) free_[0] = bytes / 256 * 256;
    }
    void* alloc(size_t bytes) {
        bytes = align_up(std::max<size_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, left = it->second - bytes;
                free_.erase(it);
                if (left) free_[off + bytes] = left;
                used_[off] = bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(void* p) {
        if (!p) return;
        const size_t off = static_cast<unsigned char*>(p) - base_;
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }

  private:
    unsigned char* base_ = nullptr;
    std::map<size_t, size_t> free_;  // offset -> bytes
    std::map<size_t, size_t> used_;
};

struct Request {
    uint64_t ticket;
    rs_request req;
    size_t footprint;  // in + out + workspace bytes counted against the budget
    double t_arrive, t_start, t_done;
    rs_status status;
    bool done;
};

struct Slot {  // one launch in flight
    bool busy = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<uint64_t> tickets;
    std::vector<void*> pool_blocks;
    size_t footprint = 0;
    uint64_t* h_offsets = nullptr;  // pinned, max_batch + 1 entries
    uint32_t* h_status = nullptr;   // pinned: the device status word of the launch's workspace
};

// Bucket requests are batched when they use the default bucket count
// (max(1, n / 16), what the segmented bucket sort gives every segment).
bool default_buckets(const rs_request& r) {
    return r.num_buckets == 0 || r.num_buckets == std::max<size_t>(1, r.n / 16);
}

// Requests that one segmented call can sort together: same algorithm, key
// width, value presence, and key_bits (radix) or declared bounds (bucket:
// the same [min, max], or bounds computed for each).
bool batch_compatible(const rs_request& a, const rs_request& b) {
    if (a.algo != b.algo || a.key_bytes != b.key_bytes || (a.vals_in != nullptr) != (b.vals_in != nullptr))
        return false;
    if (a.algo == RS_ALGO_RADIX) return a.key_bits == b.key_bits;
    const bool ca = a.min_key > a.max_key, cb = b.min_key > b.max_key;
    return default_buckets(a) && default_buckets(b) && (ca ? cb : (!cb && a.min_key == b.min_key &&
                                                                   a.max_key == b.max_key));
}

size_t batch_ws_bytes(const rs_request& q0, size_t keys, size_t count) {
    const bool vals = q0.vals_in != nullptr;
    return q0.algo == RS_ALGO_BUCKET ? seg_bucket_workspace_bytes(q0.key_bytes, vals, keys, count, 16)
                                     : segmented_workspace_bytes(q0.key_bytes, vals, keys, count, q0.key_bits);
}

size_t request_ws_bytes(const rs_request& r) {
    const bool vals = r.vals_in != nullptr;
    if (r.algo == RS_ALGO_BUCKET) return bucket_workspace_bytes(r.key_bytes, vals, r.n, r.num_buckets);
    return rs_workspace_bytes(RS_ALGO_RADIX, r.key_bytes, vals, r.n, r.key_bits, 0, 0);
}

}  // namespace

struct ServerImpl {
    rs_server_config cfg{};
    PoolAllocator pool;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;  // arrival order
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    size_t in_use = 0, max_in_use = 0;
    size_t max_queued = 0;  // longest the queue of waiting requests has been
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_requests = 0;
    bool stopping = false, cancel = false;
    std::thread worker;
    int device = 0;

    void run();
    bool launch_single(Slot& s, Request& r);
    bool launch_batch(Slot& s, std::vector<Request*>& batch, size_t footprint);
    void finish_slot(Slot& s, rs_status st);
};

// Completes every request of a slot.  A launch that ran reports the status
// word of its workspace (copied to h_status behind the sort), so errors found
// on the device (a key outside the declared range, a bounded wait that gave
// up) reach the request instead of an RS_OK with unspecified output.
void ServerImpl::finish_slot(Slot& s, rs_status st) {
    const double t = now_ms();
    if (st == RS_OK && s.h_status && *s.h_status != 0u) st = static_cast<rs_status>(*s.h_status);
    for (uint64_t tk : s.tickets) {
        auto it = reqs.find(tk);
        if (it == reqs.end()) continue;
        it->second.t_done = t;
        it->second.status = st;
        it->second.done = true;
        ++completed;
    }
    for (void* p : s.pool_blocks) pool.release(p);
    in_use -= s.footprint;
    s.tickets.clear();
    s.pool_blocks.clear();
    s.footprint = 0;
    s.busy = false;
}

bool ServerImpl::launch_single(Slot& s, Request& r) {
    const rs_request& q = r.req;
    const size_t wsb = request_ws_bytes(q);
    void* ws = pool.alloc(wsb);
    if (!ws) return false;
    *s.h_status = 0u;  // the slot is free: no copy into it is in flight
    rs_status st;
    const bool u32 = q.key_bytes == 4;
    if (q.algo == RS_ALGO_BUCKET)
        st = u32 ? bs_sort_u32(static_cast<const uint32_t*>(q.keys_in), static_cast<uint32_t*>(q.keys_out), q.vals_in,
                               q.vals_out, q.n, (uint32_t)q.min_key, (uint32_t)q.max_key, q.num_buckets, ws, wsb,
                               s.stream)
                 : bs_sort_u64(static_cast<const uint64_t*>(q.keys_in), static_cast<uint64_t*>(q.keys_out), q.vals_in,
                               q.vals_out, q.n, q.min_key, q.max_key, q.num_buckets, ws, wsb, s.stream);
    else
        st = u32 ? rs_sort_u32(static_cast<const uint32_t*>(q.keys_in), static_cast<uint32_t*>(q.keys_out), q.vals_in,
                               q.vals_out, q.n, q.key_bits, ws, wsb, s.stream)
                 : rs_sort_u64(static_cast<const uint64_t*>(q.keys_in), static_cast<uint64_t*>(q.keys_out), q.vals_in,
                               q.vals_out, q.n, q.key_bits, ws, wsb, s.stream);
    s.pool_blocks.push_back(ws);
    s.tickets.push_back(r.ticket);
    s.footprint = r.footprint;
    in_use += r.footprint;
    max_in_use = std::max(max_in_use, in_use);
    r.t_start = now_ms();
    if (st == RS_OK && cudaMemcpyAsync(s.h_status, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
        st = RS_ERR_CUDA;
    if (st != RS_OK || cudaEventRecord(s.done, s.stream) != cudaSuccess) {
        // work already enqueued on the stream may still use the pool blocks:
        // let it end before they are handed out again
        cudaStreamSynchronize(s.stream);
        finish_slot(s, st != RS_OK ? st : RS_ERR_CUDA);
        return true;
    }
    s.busy = true;
    return true;
}

// Small compatible requests (batch_compatible): keys (and values) are
// gathered into one array, sorted by one segmented radix or bucket call and
// scattered back.
bool ServerImpl::launch_batch(Slot& s, std::vector<Request*>& batch, size_t footprint) {
    const rs_request& q0 = batch[0]->req;
    const int kb = q0.key_bytes;
    const bool vals = q0.vals_in != nullptr;
    size_t total = 0;
    for (Request* r : batch) total += r->req.n;
    const size_t wsb = batch_ws_bytes(q0, total, batch.size());
    const size_t kbytes = total * kb, vbytes = vals ? total * 4 : 0;
    void* ws = pool.alloc(wsb);
    void* kin = pool.alloc(kbytes);
    void* kout = pool.alloc(kbytes);
    void* vin = vals ? pool.alloc(vbytes) : nullptr;
    void* vout = vals ? pool.alloc(vbytes) : nullptr;
    void* doff = pool.alloc((batch.size() + 1) * 8);
    if (!ws || !kin || !kout || !doff || (vals && (!vin || !vout))) {
        for (void* p : {ws, kin, kout, vin, vout, doff}) pool.release(p);
        return false;
    }
    *s.h_status = 0u;
    s.pool_blocks = {ws, kin, kout, doff};
    if (vals) {
        s.pool_blocks.push_back(vin);
        s.pool_blocks.push_back(vout);
    }
    size_t off = 0;
    bool ok = true;
    for (size_t i = 0; i < batch.size(); ++i) {
        const rs_request& q = batch[i]->req;
        s.h_offsets[i] = off;
        ok &= cudaMemcpyAsync(static_cast<unsigned char*>(kin) + off * kb, q.keys_in, q.n * kb,
                              cudaMemcpyDeviceToDevice, s.stream) == cudaSuccess;
        if (vals)
            ok &= cudaMemcpyAsync(static_cast<uint32_t*>(vin) + off, q.vals_in, q.n * 4, cudaMemcpyDeviceToDevice,
                                  s.stream) == cudaSuccess;
        off += q.n;
        s.tickets.push_back(batch[i]->ticket);
        batch[i]->t_start = now_ms();
    }
    s.h_offsets[batch.size()] = off;
    ok &= cudaMemcpyAsync(doff, s.h_offsets, (batch.size() + 1) * 8, cudaMemcpyHostToDevice, s.stream) == cudaSuccess;
    rs_status st = RS_OK;
    if (ok && q0.algo == RS_ALGO_BUCKET)
        st = kb == 4 ? bs_sort_segmented_u32(static_cast<const uint32_t*>(kin), static_cast<uint32_t*>(kout),
                                             static_cast<const uint32_t*>(vin), static_cast<uint32_t*>(vout),
                                             static_cast<const uint64_t*>(doff), batch.size(), total,
                                             (uint32_t)q0.min_key, (uint32_t)q0.max_key, 16, ws, wsb, s.stream)
                     : bs_sort_segmented_u64(static_cast<const uint64_t*>(kin), static_cast<uint64_t*>(kout),
                                             static_cast<const uint32_t*>(vin), static_cast<uint32_t*>(vout),
                                             static_cast<const uint64_t*>(doff), batch.size(), total, q0.min_key,
                                             q0.max_key, 16, ws, wsb, s.stream);
    else if (ok)
        st = kb == 4 ? rs_sort_segmented_u32(static_cast<const uint32_t*>(kin), static_cast<uint32_t*>(kout),
                                             static_cast<const uint32_t*>(vin), static_cast<uint32_t*>(vout),
                                             static_cast<const uint64_t*>(doff), batch.size(), total, q0.key_bits,
                                             ws, wsb, s.stream)
                     : rs_sort_segmented_u64(static_cast<const uint64_t*>(kin), static_cast<uint64_t*>(kout),
                                             static_cast<const uint32_t*>(vin), static_cast<uint32_t*>(vout),
                                             static_cast<const uint64_t*>(doff), batch.size(), total, q0.key_bits,
                                             ws, wsb, s.stream);
    for (size_t i = 0; ok && st == RS_OK && i < batch.size(); ++i) {
        const rs_request& q = batch[i]->req;
        const size_t o = s.h_offsets[i];
        ok &= cudaMemcpyAsync(q.keys_out, static_cast<unsigned char*>(kout) + o * kb, q.n * kb,
                              cudaMemcpyDeviceToDevice, s.stream) == cudaSuccess;
        if (vals)
            ok &= cudaMemcpyAsync(q.vals_out, static_cast<uint32_t*>(vout) + o, q.n * 4, cudaMemcpyDeviceToDevice,
                                  s.stream) == cudaSuccess;
    }
    // one status word for the whole batch: every request of it reports it
    if (ok && st == RS_OK)
        ok &= cudaMemcpyAsync(s.h_status, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, s.stream) == cudaSuccess;
    s.footprint = footprint;
    in_use += footprint;
    max_in_use = std::max(max_in_use, in_use);
    ++batches;
    batched_requests += batch.size();
    if (!ok || st != RS_OK || cudaEventRecord(s.done, s.stream) != cudaSuccess) {
        cudaStreamSynchronize(s.stream);  // enqueued copies and kernels still use the pool blocks
        finish_slot(s, st != RS_OK ? st : RS_ERR_CUDA);
        return true;
    }
    s.busy = true;
    return true;
}

// Footprint of a batch: the requests' own inputs and outputs, the gathered
// copies (input and output) and the segmented workspace.
size_t batch_footprint(const std::vector<Request*>& batch, size_t own, size_t keys) {
    const rs_request& q0 = batch[0]->req;
    const size_t per_key = (size_t)q0.key_bytes + (q0.vals_in != nullptr ? 4 : 0);
    return own + 2 * keys * per_key + batch_ws_bytes(q0, keys, batch.size()) + (batch.size() + 1) * 8;
}

void ServerImpl::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // completions
        for (Slot& s : slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaSuccess) finish_slot(s, RS_OK);
            else if (e != cudaErrorNotReady) finish_slot(s, RS_ERR_CUDA);
        }
        if (cancel && !pending.empty()) {
            const double t = now_ms();
            for (uint64_t tk : pending) {
                Request& r = reqs[tk];
                r.status = RS_ERR_SHUTDOWN;
                r.done = true;
                r.t_done = t;
            }
            pending.clear();
        }
        cv.notify_all();
        bool any_busy = std::any_of(slots.begin(), slots.end(), [](const Slot& s) { return s.busy; });
        if (stopping && pending.empty() && !any_busy) break;
        // admissions: the oldest waiting request first, into any free slot
        while (!pending.empty()) {
            auto slot_it = std::find_if(slots.begin(), slots.end(), [](const Slot& s) { return !s.busy; });
            if (slot_it == slots.end()) break;
            Request& head = reqs[pending.front()];
            const rs_request& q = head.req;
            const bool vals = q.vals_in != nullptr;
            std::vector<Request*> batch;
            size_t own = 0, keys = 0, bfp = 0;
            if (q.n <= cfg.batch_max_keys && cfg.max_batch > 1 && batch_compatible(q, q)) {
                // gather waiting small requests of the same kind, oldest first
                for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < cfg.max_batch; ++it) {
                    Request& r = reqs[*it];
                    const rs_request& x = r.req;
                    if (x.n > cfg.batch_max_keys || !batch_compatible(q, x)) continue;
                    const size_t own2 = own + 2 * x.n * ((size_t)x.key_bytes + (vals ? 4 : 0));
                    batch.push_back(&r);
                    const size_t fp2 = batch_footprint(batch, own2, keys + x.n);
                    if (in_use + fp2 > cfg.budget_bytes) {
                        batch.pop_back();
                        continue;
                    }
                    own = own2;
                    keys += x.n;
                    bfp = fp2;
                }
            }
            bool started = false;
            if (batch.size() >= 2) {
                started = launch_batch(*slot_it, batch, bfp);
                if (started)
                    for (Request* r : batch) pending.erase(std::find(pending.begin(), pending.end(), r->ticket));
            }
            if (!started) {
                if (in_use + head.footprint > cfg.budget_bytes) break;  // wait for memory to free up
                started = launch_single(*slot_it, head);
                if (started) pending.pop_front();
            }
            if (!started) {
                any_busy = std::any_of(slots.begin(), slots.end(), [](const Slot& s) { return s.busy; });
                if (!any_busy) {  // the pool cannot hold it even when idle
                    head.status = RS_ERR_BUDGET;
                    head.done = true;
                    head.t_done = now_ms();
                    ++rejected;
                    pending.pop_front();
                    continue;
                }
                break;
            }
        }
        // sleep until a request arrives or a launch may have finished
        any_busy = std::any_of(slots.begin(), slots.end(), [](const Slot& s) { return s.busy; });
        cv.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 500));
    }
    cv.notify_all();
}

}  // namespace rs

using namespace rs;

struct rs_server {
    ServerImpl impl;
};

extern "C" {

rs_status rs_server_create(const rs_server_config* cfg, rs_server** out) {
    if (!cfg || !out || !cfg->pool || cfg->pool_bytes < 4096 || cfg->num_streams < 1 || cfg->num_streams > 64 ||
        cfg->max_batch < 1 || ((uintptr_t)cfg->pool % 256))
        return RS_ERR_INVALID_ARG;
    rs_server* s = new rs_server();
    ServerImpl& m = s->impl;
    m.cfg = *cfg;
    if (m.cfg.budget_bytes == 0 || m.cfg.budget_bytes > cfg->pool_bytes) m.cfg.budget_bytes = cfg->pool_bytes;
    if (m.cfg.batch_max_keys == 0) m.cfg.batch_max_keys = 1 << 18;
    m.pool.init(cfg->pool, cfg->pool_bytes);
    if (cudaGetDevice(&m.device) != cudaSuccess) {
        delete s;
        return RS_ERR_CUDA;
    }
    m.slots.resize(cfg->num_streams);
    for (Slot& sl : m.slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_offsets, ((size_t)cfg->max_batch + 1) * 8) != cudaSuccess ||
            cudaMallocHost(&sl.h_status, sizeof(uint32_t)) != cudaSuccess) {
            for (Slot& t : m.slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
                if (t.h_offsets) cudaFreeHost(t.h_offsets);
                if (t.h_status) cudaFreeHost(t.h_status);
            }
            delete s;
            return RS_ERR_CUDA;
        }
    }
    m.worker = std::thread([&m] { m.run(); });
    *out = s;
    return RS_OK;
}

rs_status rs_server_submit(rs_server* s, const rs_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return RS_ERR_INVALID_ARG;
    const rs_request& q = *req;
    if ((q.key_bytes != 4 && q.key_bytes != 8) || (q.algo != RS_ALGO_RADIX && q.algo != RS_ALGO_BUCKET))
        return RS_ERR_INVALID_ARG;
    if (q.n == 0 || q.n > RS_MAX_KEYS || !q.keys_in || !q.keys_out || (q.vals_in == nullptr) != (q.vals_out == nullptr))
        return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    Request r{};
    r.req = q;
    if (r.req.algo == RS_ALGO_RADIX) {
        if (r.req.key_bits == 0) r.req.key_bits = 8 * q.key_bytes;
        if (r.req.key_bits < 1 || r.req.key_bits > 8 * q.key_bytes) return RS_ERR_INVALID_ARG;
    } else {
        r.req.key_bits = 8 * q.key_bytes;
        if (r.req.min_key > r.req.max_key) {  // bounds computed on the device: one marker for every key width
            r.req.min_key = 1;
            r.req.max_key = 0;
        } else if (q.key_bytes == 4 && r.req.max_key > 0xffffffffull) {
            return RS_ERR_INVALID_ARG;
        }
    }
    const size_t ws = request_ws_bytes(r.req);
    if (ws == 0) return RS_ERR_INVALID_ARG;
    r.footprint = ws + 2 * q.n * (size_t)q.key_bytes + (q.vals_in ? 2 * q.n * 4 : 0);
    std::lock_guard<std::mutex> lk(m.mu);
    if (m.stopping) return RS_ERR_SHUTDOWN;
    if (r.footprint > m.cfg.budget_bytes || ws > m.cfg.pool_bytes) {
        ++m.rejected;
        return RS_ERR_BUDGET;
    }
    r.ticket = m.next_ticket++;
    r.t_arrive = now_ms();
    r.status = RS_ERR_NOT_READY;
    m.reqs[r.ticket] = r;
    m.pending.push_back(r.ticket);
    m.max_queued = std::max(m.max_queued, m.pending.size());
    ++m.submitted;
    *ticket = r.ticket;
    m.cv.notify_all();
    return RS_OK;
}

rs_status rs_server_poll(rs_server* s, uint64_t ticket, rs_result* out) {
    if (!s) return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    std::lock_guard<std::mutex> lk(m.mu);
    auto it = m.reqs.find(ticket);
    if (it == m.reqs.end()) return RS_ERR_INVALID_ARG;
    const Request& r = it->second;
    if (out) {
        out->status = r.done ? r.status : RS_ERR_NOT_READY;
        out->t_arrive_ms = r.t_arrive;
        out->t_start_ms = r.t_start;
        out->t_done_ms = r.t_done;
    }
    return r.done ? r.status : RS_ERR_NOT_READY;
}

rs_status rs_server_release(rs_server* s, uint64_t ticket) {
    if (!s) return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    std::lock_guard<std::mutex> lk(m.mu);
    auto it = m.reqs.find(ticket);
    if (it == m.reqs.end()) return RS_ERR_INVALID_ARG;
    if (!it->second.done) return RS_ERR_NOT_READY;
    m.reqs.erase(it);
    return RS_OK;
}

rs_status rs_server_wait(rs_server* s, uint64_t ticket, int timeout_ms) {
    if (!s) return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    std::unique_lock<std::mutex> lk(m.mu);
    auto pred = [&] {
        auto it = m.reqs.find(ticket);
        return it == m.reqs.end() || it->second.done;
    };
    if (timeout_ms < 0)
        m.cv.wait(lk, pred);
    else if (!m.cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return RS_ERR_NOT_READY;
    auto it = m.reqs.find(ticket);
    if (it == m.reqs.end()) return RS_ERR_INVALID_ARG;
    return it->second.status;
}

rs_status rs_server_get_stats(rs_server* s, rs_server_stats* out) {
    if (!s || !out) return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    std::lock_guard<std::mutex> lk(m.mu);
    out->submitted = m.submitted;
    out->completed = m.completed;
    out->rejected = m.rejected;
    out->queued = m.pending.size();
    out->in_use_bytes = m.in_use;
    out->max_in_use_bytes = m.max_in_use;
    out->budget_bytes = m.cfg.budget_bytes;
    out->batches = m.batches;
    out->batched_requests = m.batched_requests;
    out->max_queued = m.max_queued;
    return RS_OK;
}

rs_status rs_server_destroy(rs_server* s, int cancel_pending) {
    if (!s) return RS_ERR_INVALID_ARG;
    ServerImpl& m = s->impl;
    {
        std::lock_guard<std::mutex> lk(m.mu);
        m.stopping = true;
        m.cancel = cancel_pending != 0;
        m.cv.notify_all();
    }
    if (m.worker.joinable()) m.worker.join();
    for (Slot& t : m.slots) {
        cudaStreamDestroy(t.stream);
        cudaEventDestroy(t.done);
        cudaFreeHost(t.h_offsets);
        cudaFreeHost(t.h_status);
    }
    delete s;
    return RS_OK;
}

}  // extern "C"
