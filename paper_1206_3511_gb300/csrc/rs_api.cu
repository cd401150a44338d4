// rs_api.cu -- library-wide C entry points: status strings, version,
// workspace sizing, the device status word, the debug hooks and the sorts of
// arrays held in host memory.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rs_segmented.h"

namespace rs {

namespace {
std::atomic<uint32_t> g_spin_limit{0};
std::atomic<int> g_stall_tile{-1};
constexpr uint32_t kDefaultSpinLimit = 1u << 21;  // polls; about a second with the back-off
}  // namespace

namespace {
// A positive integer from the environment, or `fallback` (read once by callers).
long env_long(const char* name, long fallback) {
    const char* v = std::getenv(name);
    if (!v || !*v) return fallback;
    char* end = nullptr;
    const long x = std::strtol(v, &end, 10);
    return (end && *end == '\0' && x > 0) ? x : fallback;
}
}  // namespace

uint32_t debug_spin_limit() {
    static const uint32_t env = (uint32_t)std::min<long>(env_long("RS_SPIN_LIMIT", kDefaultSpinLimit), 0x7fffffffL);
    uint32_t v = g_spin_limit.load(std::memory_order_relaxed);
    return v ? v : env;
}

int default_digit_bits() {
    static const int d = [] {
        const long x = env_long("RS_DIGIT_BITS", 8);
        return (x >= kMinDigitBits && x <= kMaxDigitBits) ? (int)x : 8;
    }();
    return d;
}

bool checked_mode() {
    static const bool on = env_long("RS_CHECKED", 0) == 1;
    return on;
}

int debug_stall_tile() { return g_stall_tile.load(std::memory_order_relaxed); }

namespace {
std::atomic<bool> g_profile{false};
std::atomic<uint64_t> g_launches{0};
struct ProfileRecord {
    const char* name;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mu;
std::vector<ProfileRecord> g_records;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

KernelScope::KernelScope(const char* name, cudaStream_t stream) : range_(name), slot_(-1), stream_(stream) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_profile.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t a = take_event(), b = take_event();
    if (!a || !b) return;
    if (cudaEventRecord(a, stream) != cudaSuccess) {
        g_event_pool.push_back(a);
        g_event_pool.push_back(b);
        return;
    }
    g_records.push_back(ProfileRecord{name, a, b});
    slot_ = (long)g_records.size() - 1;
}

KernelScope::~KernelScope() {
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if ((size_t)slot_ < g_records.size()) cudaEventRecord(g_records[slot_].stop, stream_);
}

int resident_grid_cached(const void* kern, int block, size_t smem, int (*query)(const void*, int, size_t)) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(kern, block, smem, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int grid = query(kern, block, smem) * device_sm_count();
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = grid;
    return grid;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < 64 && cache[dev]) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    if (dev < 64) cache[dev] = sms;
    return sms;
}

namespace {

// dev_buf of a host-buffer sort: the sort's workspace first (its header
// holds the status word), then the keys, the values and, for a segmented
// sort, the segment offsets.
struct HostSortLayout {
    size_t ws = 0, off_keys = 0, off_vals = 0, off_extra = 0, total = 0;
};

HostSortLayout host_sort_layout(size_t ws_bytes, int key_bytes, bool vals, size_t n, size_t extra_bytes) {
    HostSortLayout L;
    L.ws = ws_bytes;
    if (L.ws == 0) return L;
    Carver c;
    c.take(L.ws);
    L.off_keys = c.take(n * key_bytes);
    L.off_vals = vals ? c.take(n * 4) : 0;
    L.off_extra = extra_bytes ? c.take(extra_bytes) : 0;
    L.total = c.off;
    return L;
}

HostSortLayout host_sort_layout(int algo, int key_bytes, bool vals, size_t n, int key_bits, size_t nb) {
    size_t ws = 0;
    if (algo == RS_ALGO_RADIX) ws = radix_workspace_bytes(key_bytes, vals, n, key_bits);
    else if (algo == RS_ALGO_BUCKET) ws = bucket_workspace_bytes(key_bytes, vals, n, nb);
    return host_sort_layout(ws, key_bytes, vals, n, 0);
}

HostSortLayout segmented_host_layout(int key_bytes, bool vals, size_t n, size_t nseg, int key_bits) {
    return host_sort_layout(rs_segmented_workspace_bytes(key_bytes, vals ? 1 : 0, n, nseg, key_bits), key_bytes,
                            vals, n, (nseg + 1) * sizeof(uint64_t));
}

bool is_device_memory(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Checks of the host arrays that need no CUDA call.
rs_status check_host_arrays(int key_bytes, const void* hk_in, const void* hk_out, const uint32_t* hv_in,
                            const uint32_t* hv_out, size_t n) {
    if (!hk_in || !hk_out) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)hk_in | (uintptr_t)hk_out) % key_bytes) return RS_ERR_INVALID_ARG;
    const bool vals = hv_in != nullptr;
    if (vals && (((uintptr_t)hv_in | (uintptr_t)hv_out) % 4)) return RS_ERR_INVALID_ARG;
    const size_t kb = n * key_bytes, vb = n * 4;
    if (hk_in != hk_out && ranges_overlap(hk_in, kb, hk_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && hv_in != hv_out && ranges_overlap(hv_in, vb, hv_out, vb)) return RS_ERR_INVALID_ARG;
    if (vals && (ranges_overlap(hk_in, kb, hv_in, vb) || ranges_overlap(hk_in, kb, hv_out, vb) ||
                 ranges_overlap(hk_out, kb, hv_in, vb) || ranges_overlap(hk_out, kb, hv_out, vb)))
        return RS_ERR_INVALID_ARG;
    return RS_OK;
}

// Copy in, sort in place on the device, copy out; all on `stream`.  The
// caller has checked every argument that needs no CUDA call.  h_extra (the
// segment offsets of a segmented sort, or null) is copied in too.  `sort`
// runs the device sort on (keys, values, extra, workspace, workspace bytes).
template <class DeviceSort>
rs_status host_sort(int key_bytes, const void* hk_in, void* hk_out, const uint32_t* hv_in, uint32_t* hv_out,
                    size_t n, const HostSortLayout& L, void* buf, size_t buf_bytes, cudaStream_t stream,
                    DeviceSort sort, const void* h_extra = nullptr, size_t extra_bytes = 0) {
    const bool vals = hv_in != nullptr;
    if (is_device_memory(hk_in) || is_device_memory(hk_out) ||
        (vals && (is_device_memory(hv_in) || is_device_memory(hv_out))) || (h_extra && is_device_memory(h_extra)))
        return RS_ERR_INVALID_ARG;
    if (!buf || ((uintptr_t)buf % 256)) return RS_ERR_WORKSPACE;
    if (L.total == 0) return RS_ERR_INVALID_ARG;
    if (buf_bytes < L.total || !is_device_memory(buf)) return RS_ERR_WORKSPACE;

    unsigned char* base = static_cast<unsigned char*>(buf);
    void* dk = base + L.off_keys;
    uint32_t* dv = vals ? reinterpret_cast<uint32_t*>(base + L.off_vals) : nullptr;
    void* dx = h_extra ? base + L.off_extra : nullptr;
    const size_t kb = n * key_bytes, vb = n * 4;
    if (h_extra) RS_CUDA_TRY(cudaMemcpyAsync(dx, h_extra, extra_bytes, cudaMemcpyHostToDevice, stream));
    RS_CUDA_TRY(cudaMemcpyAsync(dk, hk_in, kb, cudaMemcpyHostToDevice, stream));
    if (vals) RS_CUDA_TRY(cudaMemcpyAsync(dv, hv_in, vb, cudaMemcpyHostToDevice, stream));
    const rs_status st = sort(dk, dv, dx, buf, L.ws);
    if (st != RS_OK) return st;
    RS_CUDA_TRY(cudaMemcpyAsync(hk_out, dk, kb, cudaMemcpyDeviceToHost, stream));
    if (vals) RS_CUDA_TRY(cudaMemcpyAsync(hv_out, dv, vb, cudaMemcpyDeviceToHost, stream));
    return RS_OK;
}

rs_status radix_host_sort(int key_bytes, const void* hk_in, void* hk_out, const uint32_t* hv_in, uint32_t* hv_out,
                          size_t n, int key_bits, void* buf, size_t buf_bytes, cudaStream_t stream) {
    const int width = 8 * key_bytes;
    if (key_bits == 0) key_bits = width;
    if (key_bits < 1 || key_bits > width) return RS_ERR_INVALID_ARG;
    if ((hv_in == nullptr) != (hv_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS) return RS_ERR_INVALID_ARG;
    if (n == 0) return RS_OK;
    const rs_status a = check_host_arrays(key_bytes, hk_in, hk_out, hv_in, hv_out, n);
    if (a != RS_OK) return a;
    const HostSortLayout L = host_sort_layout(RS_ALGO_RADIX, key_bytes, hv_in != nullptr, n, key_bits, 0);
    return host_sort(key_bytes, hk_in, hk_out, hv_in, hv_out, n, L, buf, buf_bytes, stream,
                     [&](void* dk, uint32_t* dv, void*, void* ws, size_t ws_bytes) {
                         return radix_sort_impl(key_bytes, dk, dk, dv, dv, n, key_bits, ws, ws_bytes, stream,
                                                nullptr);
                     });
}

rs_status bucket_host_sort(int key_bytes, const void* hk_in, void* hk_out, const uint32_t* hv_in, uint32_t* hv_out,
                           size_t n, uint64_t min_key, uint64_t max_key, size_t nb, void* buf, size_t buf_bytes,
                           cudaStream_t stream) {
    if ((hv_in == nullptr) != (hv_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS || nb > ((size_t)1 << 32)) return RS_ERR_INVALID_ARG;
    if (n == 0) return RS_OK;
    const rs_status a = check_host_arrays(key_bytes, hk_in, hk_out, hv_in, hv_out, n);
    if (a != RS_OK) return a;
    const HostSortLayout L = host_sort_layout(RS_ALGO_BUCKET, key_bytes, hv_in != nullptr, n, 0, nb);
    return host_sort(key_bytes, hk_in, hk_out, hv_in, hv_out, n, L, buf, buf_bytes, stream,
                     [&](void* dk, uint32_t* dv, void*, void* ws, size_t ws_bytes) {
                         return key_bytes == 4
                                    ? bs_sort_u32(static_cast<uint32_t*>(dk), static_cast<uint32_t*>(dk), dv, dv, n,
                                                  (uint32_t)min_key, (uint32_t)max_key, nb, ws, ws_bytes, stream)
                                    : bs_sort_u64(static_cast<uint64_t*>(dk), static_cast<uint64_t*>(dk), dv, dv, n,
                                                  min_key, max_key, nb, ws, ws_bytes, stream);
                     });
}

rs_status segmented_host_sort(int key_bytes, const void* hk_in, void* hk_out, const uint32_t* hv_in,
                              uint32_t* hv_out, const uint64_t* h_off, size_t nseg, size_t n, int key_bits,
                              void* buf, size_t buf_bytes, cudaStream_t stream, const rs_config* cfg) {
    const int width = 8 * key_bytes;
    if (key_bits == 0) key_bits = width;
    if (key_bits < 1 || key_bits > width) return RS_ERR_INVALID_ARG;
    if ((hv_in == nullptr) != (hv_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n == 0 || nseg == 0) return RS_OK;
    if (!h_off || ((uintptr_t)h_off % 8)) return RS_ERR_INVALID_ARG;
    const rs_status a = check_host_arrays(key_bytes, hk_in, hk_out, hv_in, hv_out, n);
    if (a != RS_OK) return a;
    const size_t ob = (nseg + 1) * sizeof(uint64_t);
    if (ranges_overlap(h_off, ob, hk_out, n * key_bytes) || (hv_out && ranges_overlap(h_off, ob, hv_out, n * 4)))
        return RS_ERR_INVALID_ARG;
    const HostSortLayout L = segmented_host_layout(key_bytes, hv_in != nullptr, n, nseg, key_bits);
    return host_sort(
        key_bytes, hk_in, hk_out, hv_in, hv_out, n, L, buf, buf_bytes, stream,
        [&](void* dk, uint32_t* dv, void* dx, void* ws, size_t ws_bytes) {
            const uint64_t* d_off = static_cast<const uint64_t*>(dx);
            return key_bytes == 4
                       ? rs_sort_segmented_u32_ex(static_cast<uint32_t*>(dk), static_cast<uint32_t*>(dk), dv, dv,
                                                  d_off, nseg, n, key_bits, ws, ws_bytes, stream, cfg)
                       : rs_sort_segmented_u64_ex(static_cast<uint64_t*>(dk), static_cast<uint64_t*>(dk), dv, dv,
                                                  d_off, nseg, n, key_bits, ws, ws_bytes, stream, cfg);
        },
        h_off, ob);
}

}  // namespace

}  // namespace rs

using namespace rs;

extern "C" {

size_t rs_host_sort_bytes(int algo, int key_bytes, int has_values, size_t n, int key_bits, size_t num_buckets) {
    if (key_bytes != 4 && key_bytes != 8) return 0;
    if (key_bits == 0) key_bits = 8 * key_bytes;
    if (key_bits < 1 || key_bits > 8 * key_bytes || n > RS_MAX_KEYS) return 0;
    if (num_buckets > ((size_t)1 << 32)) return 0;
    return host_sort_layout(algo, key_bytes, has_values != 0, n, key_bits, num_buckets).total;
}

rs_status rs_sort_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out, const uint32_t* h_vals_in,
                           uint32_t* h_vals_out, size_t n, int key_bits, void* dev_buf, size_t dev_buf_bytes,
                           rs_stream_t stream) {
    return radix_host_sort(4, h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, key_bits, dev_buf, dev_buf_bytes,
                           stream);
}

rs_status rs_sort_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out, const uint32_t* h_vals_in,
                           uint32_t* h_vals_out, size_t n, int key_bits, void* dev_buf, size_t dev_buf_bytes,
                           rs_stream_t stream) {
    return radix_host_sort(8, h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, key_bits, dev_buf, dev_buf_bytes,
                           stream);
}

rs_status bs_sort_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out, const uint32_t* h_vals_in,
                           uint32_t* h_vals_out, size_t n, uint32_t min_key, uint32_t max_key, size_t num_buckets,
                           void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream) {
    return bucket_host_sort(4, h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, min_key, max_key, num_buckets,
                            dev_buf, dev_buf_bytes, stream);
}

rs_status bs_sort_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out, const uint32_t* h_vals_in,
                           uint32_t* h_vals_out, size_t n, uint64_t min_key, uint64_t max_key, size_t num_buckets,
                           void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream) {
    return bucket_host_sort(8, h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, min_key, max_key, num_buckets,
                            dev_buf, dev_buf_bytes, stream);
}

size_t rs_segmented_host_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg, int key_bits) {
    if (key_bytes != 4 && key_bytes != 8) return 0;
    if (key_bits == 0) key_bits = 8 * key_bytes;
    if (key_bits < 1 || key_bits > 8 * key_bytes) return 0;
    return segmented_host_layout(key_bytes, has_values != 0, n_total, nseg, key_bits).total;
}

rs_status rs_sort_segmented_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out, const uint32_t* h_vals_in,
                                     uint32_t* h_vals_out, const uint64_t* h_seg_offsets, size_t nseg,
                                     size_t n_total, int key_bits, void* dev_buf, size_t dev_buf_bytes,
                                     rs_stream_t stream, const rs_config* cfg) {
    return segmented_host_sort(4, h_keys_in, h_keys_out, h_vals_in, h_vals_out, h_seg_offsets, nseg, n_total,
                               key_bits, dev_buf, dev_buf_bytes, stream, cfg);
}

rs_status rs_sort_segmented_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out, const uint32_t* h_vals_in,
                                     uint32_t* h_vals_out, const uint64_t* h_seg_offsets, size_t nseg,
                                     size_t n_total, int key_bits, void* dev_buf, size_t dev_buf_bytes,
                                     rs_stream_t stream, const rs_config* cfg) {
    return segmented_host_sort(8, h_keys_in, h_keys_out, h_vals_in, h_vals_out, h_seg_offsets, nseg, n_total,
                               key_bits, dev_buf, dev_buf_bytes, stream, cfg);
}

const char* rs_status_string(rs_status s) {
    switch (s) {
        case RS_OK: return "RS_OK";
        case RS_ERR_INVALID_ARG: return "RS_ERR_INVALID_ARG: invalid argument";
        case RS_ERR_WORKSPACE: return "RS_ERR_WORKSPACE: workspace missing, misaligned or too small";
        case RS_ERR_KEY_RANGE: return "RS_ERR_KEY_RANGE: a key was outside the declared key range";
        case RS_ERR_BUDGET: return "RS_ERR_BUDGET: request can never fit the memory budget";
        case RS_ERR_CUDA: return "RS_ERR_CUDA: a CUDA runtime call failed";
        case RS_ERR_DEVICE_TIMEOUT: return "RS_ERR_DEVICE_TIMEOUT: a bounded inter-block wait gave up";
        case RS_ERR_NOT_READY: return "RS_ERR_NOT_READY: request still running";
        case RS_ERR_SHUTDOWN: return "RS_ERR_SHUTDOWN: request cancelled by shutdown";
        case RS_ERR_UNSUPPORTED: return "RS_ERR_UNSUPPORTED: configuration not compiled";
        case RS_ERR_CHECK_FAILED: return "RS_ERR_CHECK_FAILED: checked mode found an output out of order";
    }
    return "unknown rs_status";
}

int rs_version(void) { return 100; }

size_t rs_workspace_bytes(int algo, int key_bytes, int has_values, size_t n, int key_bits, size_t num_buckets,
                          int in_place) {
    (void)in_place;  // the radix workspace always holds one ping-pong buffer
    (void)num_buckets;
    if (key_bytes != 4 && key_bytes != 8) return 0;
    if (key_bits == 0) key_bits = 8 * key_bytes;
    if (key_bits < 1 || key_bits > 8 * key_bytes) return 0;
    if (n > RS_MAX_KEYS) return 0;
    if (algo == RS_ALGO_RADIX) return radix_workspace_bytes(key_bytes, has_values != 0, n, key_bits);
    if (algo == RS_ALGO_BUCKET) return bucket_workspace_bytes(key_bytes, has_values != 0, n, num_buckets);
    return 0;
}

size_t rs_workspace_bytes_cfg(int key_bytes, int has_values, size_t n, int key_bits, const rs_config* cfg) {
    if ((key_bytes != 4 && key_bytes != 8) || !cfg) return 0;
    if (key_bits == 0) key_bits = 8 * key_bytes;
    if (key_bits < 1 || key_bits > 8 * key_bytes || n > RS_MAX_KEYS) return 0;
    if (cfg->digit_bits < kMinDigitBits || cfg->digit_bits > kMaxDigitBits) return 0;
    return radix_workspace_bytes_cfg(key_bytes, has_values != 0, n, key_bits, *cfg);
}

rs_status rs_get_status(const void* ws, rs_stream_t stream) {
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return RS_ERR_CUDA;
    uint32_t word = 0;
    const WsHeader* h = static_cast<const WsHeader*>(ws);
    if (cudaMemcpy(&word, &h->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return RS_ERR_CUDA;
    if (word != 0 && cudaMemset(const_cast<uint32_t*>(&h->status), 0, sizeof(uint32_t)) != cudaSuccess)
        return RS_ERR_CUDA;
    return static_cast<rs_status>(word);
}

void rs_profile_enable(int enable) { g_profile.store(enable != 0, std::memory_order_relaxed); }

uint64_t rs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int rs_profile_read(rs_kernel_stat* out, int cap) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<std::string, std::pair<uint64_t, double>> acc;
    std::vector<std::string> order;
    bool failed = false;
    for (const ProfileRecord& r : g_records) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.stop) != cudaSuccess || cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess)
            failed = true;
        auto it = acc.find(r.name);
        if (it == acc.end()) {
            order.push_back(r.name);
            it = acc.emplace(r.name, std::make_pair(0ull, 0.0)).first;
        }
        it->second.first += 1;
        it->second.second += ms;
        g_event_pool.push_back(r.start);
        g_event_pool.push_back(r.stop);
    }
    g_records.clear();
    if (failed) return -1;
    int k = 0;
    for (const std::string& name : order) {
        if (k >= cap || !out) break;
        std::memset(&out[k], 0, sizeof(rs_kernel_stat));
        std::strncpy(out[k].name, name.c_str(), sizeof(out[k].name) - 1);
        out[k].launches = acc[name].first;
        out[k].total_ms = acc[name].second;
        ++k;
    }
    return k;
}

void rs_set_debug(uint32_t spin_limit, int stall_tile) {
    g_spin_limit.store(spin_limit, std::memory_order_relaxed);
    g_stall_tile.store(stall_tile, std::memory_order_relaxed);
}

}  // extern "C"
