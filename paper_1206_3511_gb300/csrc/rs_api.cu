// rs_api.cu -- library-wide C entry points: status strings, version,
// workspace sizing, the device status word and the debug hooks.
#include <atomic>
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

uint32_t debug_spin_limit() {
    uint32_t v = g_spin_limit.load(std::memory_order_relaxed);
    return v ? v : kDefaultSpinLimit;
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

KernelScope::KernelScope(const char* name, cudaStream_t stream) : slot_(-1), stream_(stream) {
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

}  // namespace rs

using namespace rs;

extern "C" {

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
