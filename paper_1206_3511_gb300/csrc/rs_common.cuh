// rs_common.cuh -- helpers shared by the kernels and host code of the sort
// library: the workspace header, the inter-block status-word encoding,
// relaxed global loads/stores, block-wide scans and workspace carving.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdint.h>

#include "rsort.h"

namespace rs {

constexpr uint32_t kFullMask = 0xffffffffu;

// Status words of the decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", NVIDIA TR 2016).  One 32-bit
// word per (tile, digit): 2 flag bits and a 30-bit count, stored with a single
// store so a reader never sees a flag without its count.
constexpr uint32_t kFlagShift = 30;
constexpr uint32_t kFlagInvalid = 0u;
constexpr uint32_t kFlagAggregate = 1u << kFlagShift;  // count = this tile's digit count
constexpr uint32_t kFlagPrefix = 2u << kFlagShift;     // count = inclusive prefix over tiles
constexpr uint32_t kCountMask = (1u << kFlagShift) - 1u;

constexpr int kMinDigitBits = 4;
constexpr int kMaxDigitBits = 11;
constexpr int kMaxPasses = 16;  // 64-bit keys at 4-bit digits

// First 256 bytes of every workspace.
struct WsHeader {
    // The whole header is zeroed at the start of every call.
    uint32_t status;        // first device error of the last call (RS_OK = none)
    uint32_t error_detail;  // tile or block index of that error, for debugging
    uint32_t unsorted;      // radix sort: nonzero once a key is found above its successor
    uint32_t reserved0[5];
    uint32_t tile_ctr[kMaxPasses];  // dynamic tile counters, one per pass
    uint32_t done_ctr[8];           // "last block" counters
    uint32_t reserved1[64 - 8 - kMaxPasses - 8];
};
static_assert(sizeof(WsHeader) == 256, "workspace header must be 256 bytes");

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Shared-memory accesses through 32-bit shared-window addresses, with the
// predicate inside the instruction (no branch around the access).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_or_shared_if(uint32_t addr, uint32_t v, bool pred) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %2, 0; @p red.shared.or.b32 [%0], %1; }" ::"r"(addr), "r"(v),
        "r"((uint32_t)pred)
        : "memory");
}

__device__ __forceinline__ uint2 ld_shared_v2(uint32_t addr) {
    uint2 r;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(addr) : "memory");
    return r;
}

__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t r;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(addr) : "memory");
    return r;
}

__device__ __forceinline__ void st_shared_v2_if(uint32_t addr, uint32_t x, uint32_t y, bool pred) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %3, 0; @p st.shared.v2.u32 [%0], {%1, %2}; }" ::"r"(addr), "r"(x), "r"(y),
        "r"((uint32_t)pred)
        : "memory");
}

__device__ __forceinline__ void st_shared_u32_if(uint32_t addr, uint32_t v, bool pred) {
    asm volatile(
        "{ .reg .pred p; setp.ne.u32 p, %2, 0; @p st.shared.u32 [%0], %1; }" ::"r"(addr), "r"(v), "r"((uint32_t)pred)
        : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_device_error(WsHeader* h, uint32_t code, uint32_t detail) {
    if (atomicCAS(&h->status, 0u, code) == 0u) h->error_detail = detail;
}

// Order-preserving bijection from a key type to unsigned integers of the same
// width: a signed key flips its sign bit; an IEEE-754 float flips its sign bit
// when it is non-negative and every bit when it is negative (the unsigned
// order of the result is the standard's totalOrder: -NaN < -inf < ... < -0 <
// +0 < ... < +inf < +NaN); a descending sort complements the result.  Radix
// digits are taken from to_ordered(key); the sorted keys are written back
// through from_ordered.
enum KeyKind : int { kKindUnsigned = 0, kKindSigned = 1, kKindFloat = 2 };

struct KeyXform {
    int kind;
    int descending;
    __host__ __device__ __forceinline__ bool active() const { return kind != kKindUnsigned || descending; }
    template <typename KeyT>
    __host__ __device__ __forceinline__ KeyT to_ordered(KeyT k) const {
        constexpr KeyT top = (KeyT)1 << (8 * sizeof(KeyT) - 1);
        if (kind == kKindSigned) k ^= top;
        else if (kind == kKindFloat) k ^= (k & top) ? (KeyT)~(KeyT)0 : top;
        return descending ? (KeyT)~k : k;
    }
    template <typename KeyT>
    __host__ __device__ __forceinline__ KeyT from_ordered(KeyT y) const {
        constexpr KeyT top = (KeyT)1 << (8 * sizeof(KeyT) - 1);
        if (descending) y = (KeyT)~y;
        if (kind == kKindSigned) y ^= top;
        else if (kind == kKindFloat) y ^= (y & top) ? top : (KeyT)~(KeyT)0;
        return y;
    }
};

// Exclusive prefix sum of one value per thread across the block.  s_warp needs
// BLOCK/32 + 1 words; the block total lands in s_warp[BLOCK/32].  Contains
// __syncthreads() and must be reached by every thread.  Without TAIL_SYNC
// the caller must pass another barrier before s_warp is written again.
template <int BLOCK, bool TAIL_SYNC = true>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t* s_warp) {
    constexpr int kWarps = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kWarps ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFullMask, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kWarps) s_warp[lane] = wi - w;
        if (lane == kWarps - 1) s_warp[kWarps] = wi;
    }
    __syncthreads();
    uint32_t r = inc - x + s_warp[warp];
    if (TAIL_SYNC) __syncthreads();  // s_warp may be written again at once
    return r;
}

// In-place exclusive prefix sum of a[0..len) in shared memory; each thread
// scans a contiguous run of ceil(len/BLOCK) entries.
template <int BLOCK>
__device__ __forceinline__ void block_exclusive_scan_smem(uint32_t* a, int len, uint32_t* s_warp) {
    const int per = (len + BLOCK - 1) / BLOCK;
    const int start = threadIdx.x * per;
    uint32_t sum = 0;
    for (int i = 0; i < per; ++i) {
        int j = start + i;
        if (j < len) sum += a[j];
    }
    uint32_t run = block_exclusive_sum<BLOCK>(sum, s_warp);
    for (int i = 0; i < per; ++i) {
        int j = start + i;
        if (j < len) {
            uint32_t v = a[j];
            a[j] = run;
            run += v;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- host side
__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Hands out 256-byte aligned regions of a workspace in order.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off += align_up(bytes, 256);
        return o;
    }
};

inline bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
    if (!a || !b || !abytes || !bbytes) return false;
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bbytes && y < x + abytes;
}

// Library-wide debug knobs (rs_set_debug; the environment variable
// RS_SPIN_LIMIT sets the spin limit when rs_set_debug has not).
uint32_t debug_spin_limit();
int debug_stall_tile();
int device_sm_count();

// Digit width of radix sorts that name no kernel shape: 8, or the
// environment variable RS_DIGIT_BITS (4 .. 11) read once.
int default_digit_bits();

// Checked mode (environment variable RS_CHECKED=1, read once): rs_sort_*,
// rs_sort_typed and bs_sort_* verify on the device that their output is in
// nondecreasing order and record RS_ERR_CHECK_FAILED otherwise.
bool checked_mode();

// A named NVTX range on the host timeline (nvtxRangePush / Pop) for as long
// as the object lives; without a profiler attached it costs one test.
class NvtxRange {
  public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Wraps one kernel launch: counts it and, while rs_profile_enable(1) is in
// force, records CUDA events around it on its stream.
class KernelScope {
  public:
    KernelScope(const char* name, cudaStream_t stream);
    ~KernelScope();
    KernelScope(const KernelScope&) = delete;
    KernelScope& operator=(const KernelScope&) = delete;

  private:
    NvtxRange range_;
    long slot_;
    cudaStream_t stream_;
};

#define RS_CUDA_TRY(expr)                           \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return RS_ERR_CUDA;  \
    } while (0)

}  // namespace rs
