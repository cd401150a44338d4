// rs_plan.cu -- plans: one sort call with fixed buffers and sizes, captured
// once into a CUDA graph and replayed with one host launch.  For radix sorts
// the plan can first autotune the kernel shape (digit width, threads per
// block, keys per thread) by timing every compiled shape that fits the
// workspace; every shape gives bit-identical output, so tuning changes only
// the speed.  Tuning results are cached per (GPU, key width, values, key
// bits, log2 n).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rs_segmented.h"

namespace rs {

rs_status radix_sort_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                          uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                          cudaStream_t stream, const rs_config* cfg);

namespace {

rs_status enqueue_plan(const rs_plan_desc& d, const rs_config* cfg, cudaStream_t s) {
    switch (d.algo) {
        case RS_PLAN_RADIX:
            return radix_sort_impl(d.key_bytes, d.keys_in, d.keys_out, d.vals_in, d.vals_out, d.n, d.key_bits, d.ws,
                                   d.ws_bytes, s, cfg);
        case RS_PLAN_BUCKET:
            return d.key_bytes == 4
                       ? bs_sort_u32(static_cast<const uint32_t*>(d.keys_in), static_cast<uint32_t*>(d.keys_out),
                                     d.vals_in, d.vals_out, d.n, (uint32_t)d.min_key, (uint32_t)d.max_key,
                                     d.num_buckets, d.ws, d.ws_bytes, s)
                       : bs_sort_u64(static_cast<const uint64_t*>(d.keys_in), static_cast<uint64_t*>(d.keys_out),
                                     d.vals_in, d.vals_out, d.n, d.min_key, d.max_key, d.num_buckets, d.ws,
                                     d.ws_bytes, s);
        case RS_PLAN_SEGMENTED:
            return d.key_bytes == 4
                       ? rs_sort_segmented_u32_ex(static_cast<const uint32_t*>(d.keys_in),
                                                  static_cast<uint32_t*>(d.keys_out), d.vals_in, d.vals_out,
                                                  d.d_seg_offsets, d.nseg, d.n, d.key_bits, d.ws, d.ws_bytes, s, cfg)
                       : rs_sort_segmented_u64_ex(static_cast<const uint64_t*>(d.keys_in),
                                                  static_cast<uint64_t*>(d.keys_out), d.vals_in, d.vals_out,
                                                  d.d_seg_offsets, d.nseg, d.n, d.key_bits, d.ws, d.ws_bytes, s, cfg);
    }
    return RS_ERR_INVALID_ARG;
}

using TuneKey = std::tuple<std::string, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, rs_config> g_tune_cache;

TuneKey tune_key(const rs_plan_desc& d) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    const int kbits = d.key_bits ? d.key_bits : 8 * d.key_bytes;
    return TuneKey(std::string(prop.name), d.algo, d.key_bytes, d.vals_in != nullptr, kbits,
                   d.n ? (int)std::floor(std::log2((double)d.n)) : 0);
}

// ---------------------------------------------------------------- persisted tuning results
// A tuning cache file holds one JSON object per line:
//   {"gpu": "NVIDIA GB300", "algo": 0, "key_bytes": 4, "values": 0,
//    "key_bits": 32, "log2n": 26, "digit_bits": 8, "block_threads": 256,
//    "items_per_thread": 22}
// Lines that do not parse, or name a shape this build does not compile, are
// skipped.  The environment variable RS_TUNE_CACHE names a file that plans
// read before their first tuning and rewrite after every new result.

// The value after "name": in a line (a string without quotes, or a number).
bool json_field(const std::string& line, const char* name, std::string* out) {
    const std::string key = std::string("\"") + name + "\"";
    size_t p = line.find(key);
    if (p == std::string::npos) return false;
    p = line.find(':', p + key.size());
    if (p == std::string::npos) return false;
    ++p;
    while (p < line.size() && line[p] == ' ') ++p;
    if (p < line.size() && line[p] == '"') {
        const size_t q = line.find('"', p + 1);
        if (q == std::string::npos) return false;
        *out = line.substr(p + 1, q - p - 1);
        return true;
    }
    size_t q = p;
    while (q < line.size() && (line[q] == '-' || (line[q] >= '0' && line[q] <= '9'))) ++q;
    if (q == p) return false;
    *out = line.substr(p, q - p);
    return true;
}

bool json_int(const std::string& line, const char* name, int* out) {
    std::string v;
    if (!json_field(line, name, &v)) return false;
    char* end = nullptr;
    const long x = std::strtol(v.c_str(), &end, 10);
    if (!end || *end != '\0' || x < -1000000 || x > 1000000) return false;
    *out = (int)x;
    return true;
}

// A shape is usable for a key if this build compiles it for that algorithm.
bool shape_compiled(int algo, int key_bytes, bool vals, const rs_config& c) {
    if (algo == RS_PLAN_SEGMENTED)
        return c.digit_bits == kSegDigitBits && seg_shape_find(key_bytes, vals, c.block_threads, c.items_per_thread) >= 0;
    if (algo != RS_PLAN_RADIX || c.digit_bits < kMinDigitBits || c.digit_bits > kMaxDigitBits) return false;
    const Variant* v = find_variant(key_bytes, vals, c.block_threads, c.items_per_thread);
    return v && v->smem_bytes(c.digit_bits) <= kMaxSmemPerBlock;
}

bool parse_tune_line(const std::string& line, TuneKey* key, rs_config* cfg) {
    std::string gpu;
    int algo, kb, vals, kbits, l2n;
    if (!json_field(line, "gpu", &gpu) || !json_int(line, "algo", &algo) || !json_int(line, "key_bytes", &kb) ||
        !json_int(line, "values", &vals) || !json_int(line, "key_bits", &kbits) || !json_int(line, "log2n", &l2n) ||
        !json_int(line, "digit_bits", &cfg->digit_bits) || !json_int(line, "block_threads", &cfg->block_threads) ||
        !json_int(line, "items_per_thread", &cfg->items_per_thread))
        return false;
    if ((kb != 4 && kb != 8) || (vals != 0 && vals != 1) || kbits < 1 || kbits > 8 * kb || l2n < 0 || l2n > 40)
        return false;
    if (!shape_compiled(algo, kb, vals != 0, *cfg)) return false;
    *key = TuneKey(gpu, algo, kb, vals, kbits, l2n);
    return true;
}

std::string tune_line(const TuneKey& k, const rs_config& c) {
    std::string gpu = std::get<0>(k);
    for (char& ch : gpu)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 0x20) ch = '_';
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "{\"gpu\": \"%s\", \"algo\": %d, \"key_bytes\": %d, \"values\": %d, \"key_bits\": %d, "
                  "\"log2n\": %d, \"digit_bits\": %d, \"block_threads\": %d, \"items_per_thread\": %d}",
                  gpu.c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                  c.digit_bits, c.block_threads, c.items_per_thread);
    return buf;
}

// Merge a cache file into the in-process cache: entries read, or -1.
int tune_cache_load_locked(const char* path) {
    std::ifstream f(path);
    if (!f) return -1;
    int got = 0;
    std::string line;
    while (std::getline(f, line)) {
        TuneKey k;
        rs_config c{};
        if (parse_tune_line(line, &k, &c)) {
            g_tune_cache[k] = c;
            ++got;
        }
    }
    return got;
}

// Write the in-process cache (through a temporary file renamed over the
// target, so a reader never sees half a file): entries written, or -1.
int tune_cache_save_locked(const char* path) {
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return -1;
        for (const auto& e : g_tune_cache) f << tune_line(e.first, e.second) << "\n";
        if (!f) return -1;
    }
    if (std::rename(tmp.c_str(), path) != 0) return -1;
    return (int)g_tune_cache.size();
}

const char* env_tune_cache() {
    const char* p = std::getenv("RS_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// Time one shape: mean of `reps` runs after one warm-up run.
float time_config(const rs_plan_desc& d, const rs_config& cfg, cudaStream_t s, cudaEvent_t a, cudaEvent_t b,
                  int reps) {
    if (enqueue_plan(d, &cfg, s) != RS_OK) return -1.f;
    cudaEventRecord(a, s);
    for (int r = 0; r < reps; ++r)
        if (enqueue_plan(d, &cfg, s) != RS_OK) return -1.f;
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) return -1.f;
    if (rs_get_status(d.ws, s) != RS_OK) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms / reps;
}

// The shape a plan uses without tuning: the radix default, or the default
// segmented shape at 8-bit digits.
rs_status default_shape(const rs_plan_desc& d, rs_config* out) {
    if (d.algo == RS_PLAN_SEGMENTED) {
        out->digit_bits = kSegDigitBits;
        return seg_shape_get(d.key_bytes, d.vals_in != nullptr, 0, &out->block_threads, &out->items_per_thread)
                   ? RS_OK
                   : RS_ERR_UNSUPPORTED;
    }
    return rs_default_config(d.key_bytes, d.vals_in != nullptr, d.n, out);
}

rs_status autotune(const rs_plan_desc& d, cudaStream_t s, rs_config* best, float* best_ms) {
    const TuneKey key = tune_key(d);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        static bool env_loaded = false;
        if (!env_loaded) {
            env_loaded = true;
            if (const char* p = env_tune_cache()) tune_cache_load_locked(p);
        }
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second;
            *best_ms = -1.f;
            return RS_OK;
        }
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return RS_ERR_CUDA;
    const int kbits = d.key_bits ? d.key_bits : 8 * d.key_bytes;
    const bool vals = d.vals_in != nullptr;
    const bool seg = d.algo == RS_PLAN_SEGMENTED;
    const int count = seg ? seg_shape_count(d.key_bytes, vals) : rs_config_count(d.key_bytes, vals);
    float found = -1.f;
    for (int i = 0; i < count; ++i) {
        rs_config c{};
        if (seg) {
            // segmented passes: every compiled shape at 8-bit digits, one workspace for all
            c.digit_bits = kSegDigitBits;
            if (!seg_shape_get(d.key_bytes, vals, i, &c.block_threads, &c.items_per_thread)) continue;
        } else {
            if (rs_config_get(d.key_bytes, vals, i, &c) != RS_OK) continue;
            const size_t need = rs_workspace_bytes_cfg(d.key_bytes, vals, d.n, kbits, &c);
            if (need == 0 || need > d.ws_bytes) continue;
        }
        const float ms = time_config(d, c, s, a, b, 3);
        if (ms > 0.f && (found < 0.f || ms < found)) {
            found = ms;
            *best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (found < 0.f) return default_shape(d, best);
    *best_ms = found;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = *best;
    if (const char* p = env_tune_cache()) tune_cache_save_locked(p);  // best effort: tuning stands regardless
    return RS_OK;
}

}  // namespace

}  // namespace rs

using namespace rs;

struct rs_plan {
    rs_plan_desc desc;
    rs_config cfg;
    bool has_cfg;
    float tuned_ms;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    size_t kernel_nodes;
};

extern "C" {

int rs_tune_cache_load(const char* path) {
    if (!path) return -1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return tune_cache_load_locked(path);
}

int rs_tune_cache_save(const char* path) {
    if (!path) return -1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return tune_cache_save_locked(path);
}

int rs_tune_cache_size(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int)g_tune_cache.size();
}

void rs_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
}

rs_status rs_plan_create(const rs_plan_desc* desc, rs_plan** out) {
    if (!desc || !out) return RS_ERR_INVALID_ARG;
    const rs_plan_desc& d = *desc;
    if (d.algo != RS_PLAN_RADIX && d.algo != RS_PLAN_BUCKET && d.algo != RS_PLAN_SEGMENTED) return RS_ERR_INVALID_ARG;
    if (d.key_bytes != 4 && d.key_bytes != 8) return RS_ERR_INVALID_ARG;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return RS_ERR_CUDA;
    rs_plan* p = new rs_plan();
    p->desc = d;
    p->has_cfg = false;
    p->tuned_ms = -1.f;
    rs_status st = RS_OK;
    if (d.algo == RS_PLAN_RADIX || d.algo == RS_PLAN_SEGMENTED) {
        if (d.autotune)
            st = autotune(d, s, &p->cfg, &p->tuned_ms);
        else
            st = default_shape(d, &p->cfg);
        p->has_cfg = st == RS_OK;
    }
    if (st == RS_OK) {
        // a dry enqueue outside capture checks the arguments and sets kernel attributes
        st = enqueue_plan(d, p->has_cfg ? &p->cfg : nullptr, s);
        if (st == RS_OK && cudaStreamSynchronize(s) != cudaSuccess) st = RS_ERR_CUDA;
    }
    if (st == RS_OK) {
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            st = RS_ERR_CUDA;
        } else {
            st = enqueue_plan(d, p->has_cfg ? &p->cfg : nullptr, s);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st == RS_OK && e != cudaSuccess) st = RS_ERR_CUDA;
            p->graph = g;
            if (st == RS_OK && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) st = RS_ERR_CUDA;
        }
    }
    if (st == RS_OK) {
        size_t nn = 0;
        cudaGraphGetNodes(p->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) cudaGraphGetNodes(p->graph, nodes.data(), &nn);
        for (cudaGraphNode_t node : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(node, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++p->kernel_nodes;
        }
    }
    cudaStreamDestroy(s);
    if (st != RS_OK) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return st;
    }
    *out = p;
    return RS_OK;
}

rs_status rs_plan_launch(rs_plan* plan, rs_stream_t stream) {
    if (!plan || !plan->exec) return RS_ERR_INVALID_ARG;
    return cudaGraphLaunch(plan->exec, stream) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status rs_plan_info(const rs_plan* plan, rs_config* cfg, size_t* kernel_nodes, float* tuned_ms) {
    if (!plan) return RS_ERR_INVALID_ARG;
    if (cfg) {
        if (plan->has_cfg)
            *cfg = plan->cfg;
        else
            *cfg = rs_config{0, 0, 0};
    }
    if (kernel_nodes) *kernel_nodes = plan->kernel_nodes;
    if (tuned_ms) *tuned_ms = plan->tuned_ms;
    return RS_OK;
}

void rs_plan_destroy(rs_plan* plan) {
    if (!plan) return;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
}

}  // extern "C"
