// rs_noalloc.cu -- a radix-sort entry point for callers that cannot allocate
// device memory.
//
// Some callers have no way to hand this library a workspace: code that runs
// where cudaMalloc is forbidden or unavailable (inside a custom allocator's
// own callbacks, a framework hook that must not allocate, a process whose
// memory pool is fully reserved up front), or code that simply cannot manage
// the lifetime of an extra buffer.  rs_sort_u32_noalloc serves them: it runs
// the same LSD radix sort as rs_sort_u32, but its scratch memory (the
// workspace header, digit counts, look-back status words and the ping-pong
// buffer) is one fixed array of kNoAllocScratchBytes that lives in this
// library's own device memory.  Nothing is allocated per call.
//
// Costs and limits of that choice:
//   - every GPU on which the library is loaded keeps the array until the
//     process exits, whether or not the entry point is ever called;
//   - n is capped at RS_NOALLOC_MAX_KEYS; larger sorts are rejected;
//   - all calls share the one array, so two calls that overlap on the GPU
//     (different streams, or different host threads on one stream without
//     ordering) corrupt each other's results; calls must be ordered;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) and caches it; make that first call before any
//     stream capture on that device.
#include <mutex>

#include "rs_radix.h"

namespace rs {
namespace {

// 9 MiB: the workspace of a 2^20-key uint32 key-value sort with the default
// kernel shape (8.7 MiB) rounded up.
constexpr size_t kNoAllocScratchBytes = (size_t)9 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side name of the array is not a device address).
rs_status scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RS_OK;
}

// Workspace of the largest call this entry point accepts: RS_NOALLOC_MAX_KEYS
// keys with values, 32 key bits, the default kernel shape and digit width
// (the ones a call without an explicit shape uses).
size_t noalloc_scratch_needed() {
    const Variant* v = default_variant(4, true, RS_NOALLOC_MAX_KEYS, false);
    if (!v) return ~(size_t)0;
    return radix_layout(4, true, RS_NOALLOC_MAX_KEYS, 32, default_digit_bits(), v->tile_keys, true).total;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                         uint32_t* vals_out, size_t n, int key_bits, rs_stream_t stream) {
    if (n > RS_NOALLOC_MAX_KEYS) return RS_ERR_INVALID_ARG;
    void* scratch = nullptr;
    rs_status st = scratch_for_current_device(&scratch);
    if (st != RS_OK) return st;
    // the array must hold the workspace of the largest sort accepted here,
    // with values, under every kernel shape the sort may pick
    if (noalloc_scratch_needed() > kNoAllocScratchBytes) return RS_ERR_UNSUPPORTED;
    // the sort clears the parts of the scratch that must start at zero (the
    // header, the digit counts and the first pass's status words) itself
    return radix_sort_impl(4, keys_in, keys_out, vals_in, vals_out, n, key_bits, scratch, kNoAllocScratchBytes,
                           stream, nullptr);
}
