// rs_bucket.cu -- bucket sort (Sec. 2.3, Algorithm 2) on the GPU.
//
// The paper inserts every key into bucket b(k) (range-divide), sorts each
// bucket with insertion sort and concatenates the buckets.  Here the buckets
// live in contiguous ranges of the output (their concatenation costs
// nothing), and the insert step is a stable partition by bucket id done
// most-significant bits first:
//   level 1: a one-sweep pass partitions all keys by the top (up to 8) bits of
//            their bucket id;
//   level 2: partitions still larger than one block's shared memory are
//            partitioned by the next (up to 8) bits with a segmented pass;
//   leaves:  every partition of at most 4096 keys is sorted inside one block:
//            a stable counting pass by exact bucket (the insert step), then
//            each bucket sorted by a stable rank sort that makes the
//            comparisons of insertion sort (Algorithm 1) for all keys at once;
//   overflow: a partition that is still too large when the bucket bits run
//            out (skewed keys) is radix-sorted on its keys relative to the
//            lowest key its buckets can hold, using only the bits that span;
//   constant partitions (a single possible key) need no sorting at all.
// Every step is stable, so equal keys keep their input order (Sec. 2.3 last
// paragraph), and the result equals the stable sort of the keys.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "rs_bucket.cuh"
#include "rs_segmented.h"

namespace rs {

namespace {

// ---------------------------------------------------------------- kernels
template <typename KeyT>
__global__ void __launch_bounds__(256) k_minmax(const KeyT* __restrict__ keys, size_t n, unsigned long long* mm) {
    __shared__ unsigned long long s_lo[8], s_hi[8];
    unsigned long long lo = ~0ull, hi = 0ull;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long k = (unsigned long long)__ldcs(keys + i);
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(kFullMask, lo, o), b = __shfl_xor_sync(kFullMask, hi, o);
        lo = a < lo ? a : lo;
        hi = b > hi ? b : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            lo = s_lo[w] < lo ? s_lo[w] : lo;
            hi = s_hi[w] > hi ? s_hi[w] : hi;
        }
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

// Parameters of nb buckets over [lo, hi] (the reciprocals of the exact
// bucket function, computed once).
__device__ __forceinline__ BucketParams make_bucket_params(uint64_t lo, uint64_t hi, uint64_t nb, int key_bytes) {
    const uint64_t range = hi - lo + 1;  // 0 means 2^64
    BucketParams p{};
    p.min = lo;
    p.max = hi;
    p.nb = nb;
    p.range = range;
    p.recip = (range != 0 && range <= 0x100000000ull) ? (~0ull / range) : 0ull;
    p.mul_ok = (range != 0 && nb < range) ? 1u : 0u;
    p.mul = p.mul_ok ? (uint64_t)(((unsigned __int128)nb << 64) / range) : 0ull;
    p.bbits = nb > 1 ? 64u - __clzll(nb - 1) : 0u;
    p.valid = 1u;
    return p;
}

// Bucket parameters from the declared bounds or from the reduced min/max.
__global__ void k_bucket_params(BucketParams* bp, const unsigned long long* mm, uint64_t min_key, uint64_t max_key,
                                uint64_t nb, int key_bytes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *bp = make_bucket_params(mm ? mm[0] : min_key, mm ? mm[1] : max_key, nb, key_bytes);
}

// Count of every bucket (exact bucket ids, Algorithm 2's insert step without
// the lists): one global atomic per key; keys outside [min, max] are
// reported in the status word.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_bucket_counts(const KeyT* __restrict__ keys, size_t n,
                                                       const BucketParams* bpp, uint32_t* counts, WsHeader* hdr) {
    const BucketParams bp = load_bucket_params(bpp);
    bool bad = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const KeyT k = keys[i];
        if (!key_in_bounds(bp, k)) {
            bad = true;
            continue;
        }
        atomicAdd(&counts[bucket_of(bp, k)], 1u);
    }
    if (bad) set_device_error(hdr, RS_ERR_KEY_RANGE, blockIdx.x);
}

// Range check of the declared bounds in the level-1 counting kernel.
struct BucketCountDigits {
    static constexpr bool kBytesCapable = false;
    static constexpr bool kOneDigit = true;
    const BucketParams* src;
    int shift;
    uint32_t mask;
    BucketParams bp;
    __device__ __forceinline__ void init() { bp = load_bucket_params(src); }
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT k, int) const {
        return (uint32_t)(bucket_of(bp, k) >> shift) & mask;
    }
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT k) const {
        return key_in_bounds(bp, k);
    }
    template <typename KeyT>
    __device__ __forceinline__ KeyT order(KeyT k) const {
        return k;
    }
};

// ceil(b * range / nb): how many key values lie below bucket b (exact).
__device__ __forceinline__ uint64_t keys_below_bucket(const BucketParams& bp, uint64_t b) {
    if (bp.range != 0 && bp.range <= 0xffffffffull + 1 && b <= 0xffffffffull)  // b * range < 2^64
        return (b * bp.range + bp.nb - 1) / bp.nb;
    const unsigned __int128 r = bp.range ? (unsigned __int128)bp.range : ((unsigned __int128)1 << 64);
    const unsigned __int128 x = (unsigned __int128)b * r;
    return (uint64_t)((x + bp.nb - 1) / bp.nb);
}

__device__ __forceinline__ uint32_t bit_length(uint64_t x) { return x ? 64u - __clzll(x) : 0u; }

struct PlanLevel {
    const BucketParams* bp;
    int shift;        // position of this level's digit in the bucket id
    int digit_bits;   // bits of this level's digit
    // segmented bucket sort: every parent has its own parameters
    // (table[parent.grp]) and its own digit of partition level `level`; its
    // row of starts is row_stride words; at level 1 every big child goes on
    // to level 2, whatever bits are left
    const BucketParams* table;
    int level;
    uint32_t row_stride;
    uint32_t cap;     // largest partition sorted in shared memory
    uint32_t tile_keys;      // tile of the next level's partition pass
    uint32_t ovf_tile_keys;  // tile of the overflow radix passes
    // parents: either the whole array (parents == null) or a device list
    const SegDesc* parents;
    const uint32_t* num_parents;
    uint64_t n_total;          // whole-array parent size
    const uint32_t* starts;    // [parent][bins] exclusive prefixes of the digit counts
    const uint32_t* counts;    // [bins] counts (whole-array parent only)
    int in_out;                // 1: the children's keys now sit in keys_out
    int key_width;             // bits of the key type
    // outputs
    SegDesc* leaf;
    uint32_t* num_leaf;
    SegDesc* next;             // null: no further level
    SegPlanHdr* next_hdr;
    SegDesc* ovf;
    SegPlanHdr* ovf_hdr;
    SegDesc* copy;
    uint32_t* num_copy;
};

// Exclusive prefix sum of one 64-bit value per thread across the block (the
// block total in *total).  Contains __syncthreads(); every thread calls it.
template <int BLOCK>
__device__ __forceinline__ uint64_t block_exclusive_sum_u64(uint64_t x, uint64_t* s_warp, uint64_t* total) {
    constexpr int kWarps = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint64_t v = s_warp[w];
            s_warp[w] = run;
            run += v;
        }
        s_warp[kWarps] = run;
    }
    __syncthreads();
    const uint64_t r = inc - x + s_warp[warp];
    *total = s_warp[kWarps];
    __syncthreads();
    return r;
}

// One block per parent, one thread per child (digit value).  A child above
// the shared-memory capacity whose keys can differ goes to the next level
// (while bucket bits remain) or to the overflow radix; the others are
// grouped, in order, into runs of at most `cap` keys and 256 buckets, each
// sorted by one block: a run's buckets are contiguous and ordered, so sorting
// the run by bucket and then each bucket is sorting each child.  The runs
// are the greedy ones (a child joins the open run unless that would pass
// either limit); each thread finds, by binary search over prefix sums, where
// a run that starts at its child would end, and one thread follows the chain
// of run starts.  Key-value widths are carried as width - 1 so that a range
// of 2^64 values does not wrap to 0.
__global__ void __launch_bounds__(256) k_bucket_plan(PlanLevel pl) {
    constexpr int kBlock = 256;
    __shared__ uint64_t s_pn[257], s_ps[257], s_below[257];
    __shared__ uint32_t s_next[256];
    __shared__ uint8_t s_big[256], s_start[256];
    __shared__ uint64_t s_warp64[kBlock / 32 + 1];
    __shared__ uint32_t s_scan[kBlock / 32 + 1];
    __shared__ uint32_t s_valid, s_base[5];
    const uint32_t nparents = pl.parents ? *pl.num_parents : 1u;
    BucketParams bp = pl.table ? BucketParams{} : load_bucket_params(pl.bp);
    int shift = pl.shift, digit_bits = pl.digit_bits;
    const uint32_t d = threadIdx.x;
    for (uint32_t parent = blockIdx.x; parent < nparents; parent += gridDim.x) {
        uint64_t pstart = 0, pn = pl.n_total, pb_lo = 0;
        uint32_t grp = 0;
        if (pl.parents) {
            const SegDesc ps = pl.parents[parent];
            pstart = ps.start;
            pn = ps.n;
            pb_lo = ps.aux;
            grp = ps.grp;
        }
        if (pl.table) {
            bp = load_bucket_params(pl.table + grp);
            bucket_level_digit(bp.bbits, pl.level, &shift, &digit_bits);
        }
        const uint32_t bins = 1u << digit_bits;
        const bool to_next = pl.next && (pl.table ? pl.level == 1 : shift > 0);
        const uint32_t* row = pl.starts + (size_t)parent * (pl.row_stride ? pl.row_stride : bins);
        __syncthreads();
        if (d == 0) s_valid = bins;
        // this child's bucket range, keys and key values
        const uint64_t b_lo = pb_lo + ((uint64_t)d << shift);
        const bool valid = d < bins && b_lo < bp.nb;
        uint64_t off = 0, n = 0, span = 0;
        if (valid) {
            off = row[d];
            const uint64_t end = pl.counts ? off + pl.counts[d] : ((d + 1 < bins) ? row[d + 1] : pn);
            n = end > off ? end - off : 0;
            span = (uint64_t)1 << shift;
            if (span > bp.nb - b_lo) span = bp.nb - b_lo;
        }
        if (d <= bins) {
            uint64_t b = pb_lo + ((uint64_t)d << shift);
            if (b > bp.nb) b = bp.nb;
            s_below[d] = keys_below_bucket(bp, b);
        }
        if (d == 0 && bins == kBlock) {  // the entry past the last child
            uint64_t b = pb_lo + ((uint64_t)bins << shift);
            if (b > bp.nb) b = bp.nb;
            s_below[bins] = keys_below_bucket(bp, b);
        }
        __syncthreads();
        if (d < bins && !valid) atomicMin(&s_valid, d);
        uint64_t tot_n, tot_s;
        const uint64_t pn_d = block_exclusive_sum_u64<kBlock>(n, s_warp64, &tot_n);
        const uint64_t ps_d = block_exclusive_sum_u64<kBlock>(span, s_warp64, &tot_s);
        const uint32_t nvalid = s_valid;
        // width - 1 of this child's key values (valid whenever it holds a key)
        const uint64_t wm1 = valid ? s_below[d + 1] - s_below[d] - 1 : 0;
        const bool big = valid && n > pl.cap && wm1 >= 1;
        if (d < kBlock) {
            s_pn[d] = pn_d;
            s_ps[d] = ps_d;
            s_big[d] = big;
            s_start[d] = 0;
        }
        if (d == 0) {
            s_pn[kBlock] = tot_n;
            s_ps[kBlock] = tot_s;
        }
        __syncthreads();
        // where a run starting at this child ends: the first later child that
        // is big, invalid, or would take the run past cap keys or 256 buckets
        if (valid && !big) {
            uint32_t limit = d + 1;
            while (limit < nvalid && !s_big[limit]) ++limit;  // next big child (bounded by bins)
            uint32_t lo = d + 1, hi = limit;                 // the answer lies in [lo, hi]
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (s_pn[mid] - pn_d <= pl.cap && s_ps[mid] - ps_d <= 256) lo = mid;
                else hi = mid - 1;
            }
            s_next[d] = lo;
        }
        __syncthreads();
        if (d == 0) {  // follow the chain of run starts
            uint32_t st = 0;
            while (st < nvalid) {
                if (s_big[st]) {
                    ++st;
                    continue;
                }
                s_start[st] = 1;
                st = s_next[st];
            }
        }
        __syncthreads();
        // this child's outputs: a run starting here, and/or itself as a big child
        SegDesc run{}, bigc{};
        uint32_t is_leaf = 0, is_copy = 0, is_big = 0, big_tiles = 0, big_chunks = 0;
        if (valid && s_start[d]) {
            const uint32_t e = s_next[d];
            const uint64_t rn = s_pn[e] - pn_d;
            if (rn > 0) {
                const uint64_t rwm1 = s_below[e] - s_below[d] - 1;
                run.start = pstart + off;
                run.n = (uint32_t)rn;
                run.key_lo = bp.min + s_below[d];
                run.aux = b_lo;
                run.bits = rwm1 == 0 ? 0u : min(bit_length(rwm1), (uint32_t)pl.key_width);
                const uint64_t rspan = s_ps[e] - ps_d;
                run.chunk0 = rspan > 0xffffffffull ? 0xffffffffu : (uint32_t)rspan;
                run.grp = grp;
                if (run.bits == 0) is_copy = pl.in_out ? 0u : 1u;  // one possible key: in order already
                else is_leaf = 1;
            }
        }
        if (big) {
            bigc.start = pstart + off;
            bigc.n = (uint32_t)n;
            bigc.aux = b_lo;
            bigc.grp = grp;
            bigc.key_lo = to_next ? 0 : bp.min + s_below[d];  // the next level digits the key's bucket id
            bigc.bits = to_next ? 0u : min(bit_length(wm1), (uint32_t)pl.key_width);
            is_big = 1;
            big_tiles = ceil_div_u32(bigc.n, to_next ? pl.tile_keys : pl.ovf_tile_keys);
            big_chunks = ceil_div_u32(bigc.n, kSegChunk);
        }
        const uint32_t at_leaf = block_exclusive_sum<kBlock>(is_leaf, s_scan);
        const uint32_t n_leaf = s_scan[kBlock / 32];
        const uint32_t at_copy = block_exclusive_sum<kBlock>(is_copy, s_scan);
        const uint32_t n_copy = s_scan[kBlock / 32];
        const uint32_t at_big = block_exclusive_sum<kBlock>(is_big, s_scan);
        const uint32_t n_big = s_scan[kBlock / 32];
        const uint32_t at_tiles = block_exclusive_sum<kBlock>(big_tiles, s_scan);
        const uint32_t n_tiles = s_scan[kBlock / 32];
        const uint32_t at_chunks = block_exclusive_sum<kBlock>(big_chunks, s_scan);
        const uint32_t n_chunks = s_scan[kBlock / 32];
        if (d == 0) {
            SegPlanHdr* bh = to_next ? pl.next_hdr : pl.ovf_hdr;
            s_base[0] = n_leaf ? atomicAdd(pl.num_leaf, n_leaf) : 0u;
            s_base[1] = n_copy ? atomicAdd(pl.num_copy, n_copy) : 0u;
            s_base[2] = n_big ? atomicAdd(&bh->num_large, n_big) : 0u;
            s_base[3] = n_big ? atomicAdd(&bh->total_tiles, n_tiles) : 0u;
            s_base[4] = n_big ? atomicAdd(&bh->total_chunks, n_chunks) : 0u;
        }
        __syncthreads();
        if (is_leaf) pl.leaf[s_base[0] + at_leaf] = run;
        if (is_copy) pl.copy[s_base[1] + at_copy] = run;
        if (is_big) {
            bigc.tile0 = s_base[3] + at_tiles;
            bigc.chunk0 = s_base[4] + at_chunks;
            (to_next ? pl.next : pl.ovf)[s_base[2] + at_big] = bigc;
        }
    }
}

template <typename KeyT>
__global__ void __launch_bounds__(256) k_copy_segments(const KeyT* __restrict__ src_k, const uint32_t* __restrict__ src_v,
                                                       KeyT* dst_k, uint32_t* dst_v, const SegDesc* segs,
                                                       const uint32_t* count) {
    for (uint32_t si = blockIdx.x; si < *count; si += gridDim.x) {
        const SegDesc s = segs[si];
        for (uint32_t i = threadIdx.x; i < s.n; i += blockDim.x) {
            dst_k[s.start + i] = src_k[s.start + i];
            if (src_v) dst_v[s.start + i] = src_v[s.start + i];
        }
    }
}

template <typename KeyT, bool VALS>
cudaError_t launch_plain_bucket_pass(const PassParams<BucketDigit>& p, cudaStream_t s) {
    using S = BucketShape<KeyT, VALS>;
    using Shape = OnesweepShape<KeyT, VALS, S::kBlock, S::kItems>;
    auto kern = k_onesweep<KeyT, VALS, S::kBlock, S::kItems, S::kMinB, BucketDigit>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)pass_smem_bytes<Shape, BucketDigit>(8));
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t smem = pass_smem_bytes<Shape, BucketDigit>(p.digit_bits);
    const size_t grid = std::min<size_t>(p.num_tiles, (size_t)resident_grid(kern, S::kBlock, smem));
    KernelScope scope("bucket_pass", s);
    kern<<<(unsigned)(grid ? grid : 1), S::kBlock, smem, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- layout
struct BucketPlanInfo {
    int key_bytes;
    bool vals;
    size_t n, nb;
    int bbits;             // bits of the bucket id (at least 1)
    int d1, shift1;        // level 1 digit
    bool level2;
    int d2, shift2;        // level 2 digit
    int ovf_passes, ovf_bits;  // overflow radix: passes and digit bits (0 passes: none possible)
    size_t max_leaf2, max_ovf, max_tiles, max_chunks, max_rows;
};

int bit_length_host(uint64_t x) {
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

BucketPlanInfo plan_info(int key_bytes, bool vals, size_t n, size_t nb, bool bounds_known, uint64_t min_key,
                         uint64_t max_key) {
    BucketPlanInfo I{};
    I.key_bytes = key_bytes;
    I.vals = vals;
    I.n = n;
    I.nb = nb;
    I.bbits = std::max(1, bit_length_host(nb - 1));
    I.d1 = std::min(8, I.bbits);
    I.shift1 = I.bbits - I.d1;
    I.level2 = I.shift1 > 0;
    I.d2 = I.level2 ? std::min(8, I.shift1) : 0;
    I.shift2 = I.level2 ? I.shift1 - I.d2 : 0;
    // overflow partitions span 2^last_shift buckets; bound the key bits they
    // can need from the declared range (or the full key width)
    const int last_shift = I.level2 ? I.shift2 : I.shift1;
    const int width_bits = 8 * key_bytes;
    long double range = bounds_known ? (long double)(max_key - min_key) + 1.0L : std::pow(2.0L, width_bits);
    const long double span_keys = std::ceil(range * std::pow(2.0L, last_shift) / (long double)nb) + 1.0L;
    int bits = span_keys <= 1.0L ? 0 : (int)std::ceil(std::log2(span_keys));
    if (bits > width_bits) bits = width_bits;
    I.ovf_bits = 0;
    I.ovf_passes = 0;
    if (bits > 0) {
        int P = (bits + 7) / 8;
        const bool from_out = I.level2;  // overflow data sits in keys_out after level 2, else in the buffer
        if ((P % 2 == 0) != from_out) ++P;  // pass 0 must not write the array it reads
        I.ovf_passes = P;
        I.ovf_bits = (bits + P - 1) / P;
        if (I.ovf_bits < 1) I.ovf_bits = 1;
    }
    const uint32_t tk = std::min(seg_tile_keys(key_bytes, vals), bucket_tile_keys(key_bytes, vals));
    const size_t parents2 = (size_t)1 << I.d1;
    I.max_leaf2 = I.level2 ? std::min<size_t>(parents2 << I.d2, n) : 1;
    I.max_ovf = std::min<size_t>(n / kLocalCap + 1, I.level2 ? (parents2 << I.d2) : parents2);
    I.max_tiles = n / tk + std::max<size_t>(parents2, I.max_ovf) + 2;
    I.max_chunks = n / kSegChunk + std::max<size_t>(parents2, I.max_ovf) + 2;
    I.max_rows = std::max<size_t>(parents2 * 256, I.max_ovf * (size_t)std::max(1, I.ovf_passes) * 256);
    return I;
}

struct BucketLayout {
    size_t off_params, off_mm, off_hdr, off_counts1, off_scan1, off_leaf1, off_copy, off_next, off_leaf2, off_ovf,
        off_tile_seg, off_chunk_seg, off_rows, off_status0, off_status1, off_tmp_keys, off_tmp_vals, total;
};

BucketLayout bucket_layout(const BucketPlanInfo& I) {
    BucketLayout L{};
    Carver c;
    c.take(sizeof(WsHeader));
    L.off_params = c.take(sizeof(BucketParams));
    L.off_mm = c.take(16);
    L.off_hdr = c.take(4 * sizeof(SegPlanHdr));
    L.off_counts1 = c.take(256 * 4);
    L.off_scan1 = c.take(256 * 4);
    L.off_leaf1 = c.take(256 * sizeof(SegDesc));
    L.off_copy = c.take(256 * sizeof(SegDesc));
    L.off_next = c.take(256 * sizeof(SegDesc));
    L.off_leaf2 = c.take(I.max_leaf2 * sizeof(SegDesc));
    L.off_ovf = c.take(I.max_ovf * sizeof(SegDesc));
    L.off_tile_seg = c.take(I.max_tiles * 4);
    L.off_chunk_seg = c.take(I.max_chunks * 4);
    L.off_rows = c.take(I.max_rows * 4);
    L.off_status0 = c.take(I.max_tiles * 256 * 4);
    L.off_status1 = c.take(I.max_tiles * 256 * 4);
    L.off_tmp_keys = c.take(I.n * I.key_bytes);
    L.off_tmp_vals = I.vals ? c.take(I.n * 4) : 0;
    L.total = c.off;
    return L;
}

// ---------------------------------------------------------------- segmented bucket sort: kernels
// Every segment of an offsets table is bucket-sorted on its own (Algorithm 2
// per segment): its own bounds (declared for all, or its own min and max), its
// own max(1, n / keys_per_bucket) buckets.  Segment s's parameters are
// table[s]; descriptors carry s in SegDesc::grp.

// Segments of an offsets table, validated: a decreasing table, a segment
// that ends past n_total or one above the single-sort limit is reported
// (RS_ERR_INVALID_ARG) and left out.  Nonempty segments are listed in `all`
// with their min/max chunks reserved, and their min/max seeds written.
__global__ void k_segb_list(const uint64_t* __restrict__ offsets, size_t nseg, uint64_t n_total, SegDesc* all,
                            SegPlanHdr* hall, unsigned long long* mm, WsHeader* ws_hdr) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const uint64_t a = offsets[s], b = offsets[s + 1];
    if (b < a || b > n_total || b - a >= ((uint64_t)1 << 30)) {
        set_device_error(ws_hdr, RS_ERR_INVALID_ARG, (uint32_t)s);
        return;
    }
    if (!mm || b == a) return;
    mm[2 * s] = ~0ull;
    mm[2 * s + 1] = 0ull;
    SegDesc d{};
    d.start = a;
    d.n = (uint32_t)(b - a);
    d.grp = (uint32_t)s;
    d.chunk0 = atomicAdd(&hall->total_chunks, ceil_div_u32(d.n, kSegChunk));
    all[atomicAdd(&hall->num_large, 1u)] = d;
}

// chunk -> listed segment map (one block per listed segment).
__global__ void k_segb_chunk_map(const SegDesc* __restrict__ all, const SegPlanHdr* __restrict__ hall,
                                 uint32_t* chunk_seg) {
    for (uint32_t li = blockIdx.x; li < hall->num_large; li += gridDim.x) {
        const SegDesc d = all[li];
        const uint32_t nc = ceil_div_u32(d.n, kSegChunk);
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) chunk_seg[d.chunk0 + i] = li;
    }
}

// The smallest and largest key of every listed segment (b1 per segment): one
// block per counting chunk, one atomic min and max per block.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_segb_minmax(const KeyT* __restrict__ keys, const SegDesc* __restrict__ all,
                                                      const SegPlanHdr* __restrict__ hall,
                                                      const uint32_t* __restrict__ chunk_seg, unsigned long long* mm) {
    __shared__ unsigned long long s_lo[8], s_hi[8];
    for (uint32_t c = blockIdx.x; c < hall->total_chunks; c += gridDim.x) {
        const SegDesc d = all[chunk_seg[c]];
        const uint32_t lo_i = (c - d.chunk0) * kSegChunk, hi_i = min(d.n, lo_i + kSegChunk);
        unsigned long long lo = ~0ull, hi = 0ull;
        for (uint32_t i = lo_i + threadIdx.x; i < hi_i; i += 256) {
            const unsigned long long k = (unsigned long long)__ldcs(keys + d.start + i);
            lo = k < lo ? k : lo;
            hi = k > hi ? k : hi;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long x = __shfl_xor_sync(kFullMask, lo, o), y = __shfl_xor_sync(kFullMask, hi, o);
            lo = x < lo ? x : lo;
            hi = y > hi ? y : hi;
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            s_lo[threadIdx.x >> 5] = lo;
            s_hi[threadIdx.x >> 5] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; ++w) {
                lo = s_lo[w] < lo ? s_lo[w] : lo;
                hi = s_hi[w] > hi ? s_hi[w] : hi;
            }
            atomicMin(&mm[2 * d.grp], lo);
            atomicMax(&mm[2 * d.grp + 1], hi);
        }
    }
}

// Per segment: its bucket parameters, then its class.  A segment of at most
// kLocalCap keys is sorted whole by one block in bucket mode (its bucket ids
// relative to bucket 0, over its whole range); a larger one goes through the
// partition levels.  One thread per segment.
__global__ void k_segb_classify(const uint64_t* __restrict__ offsets, size_t nseg, uint64_t n_total,
                                const unsigned long long* __restrict__ mm, uint64_t min_key, uint64_t max_key,
                                uint64_t keys_per_bucket, int key_bytes, uint32_t tile_keys, BucketParams* table,
                                SegDesc* small, SegDesc* large, SegPlanHdr* hl) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const uint64_t a = offsets[s], b = offsets[s + 1];
    if (b < a || b > n_total || b - a >= ((uint64_t)1 << 30) || b == a) return;  // reported by k_segb_list
    const uint64_t n = b - a;
    const uint64_t lo = mm ? mm[2 * s] : min_key, hi = mm ? mm[2 * s + 1] : max_key;
    const uint64_t nb = n / keys_per_bucket > 0 ? n / keys_per_bucket : 1;
    const BucketParams bp = make_bucket_params(lo, hi, nb, key_bytes);
    table[s] = bp;
    SegDesc d{};
    d.start = a;
    d.n = (uint32_t)n;
    d.grp = (uint32_t)s;
    if (n <= kLocalCap) {
        d.key_lo = lo;
        d.bits = hi == lo ? 0u : 64u - __clzll(hi - lo);
        d.aux = 0;
        d.chunk0 = nb > 0xffffffffull ? 0xffffffffu : (uint32_t)nb;  // buckets the segment spans
        small[atomicAdd(&hl->num_small, 1u)] = d;
    } else {
        d.key_lo = 0;
        d.bits = 8u * (uint32_t)key_bytes;
        d.aux = 0;
        append_large(large, &hl->num_large, &hl->total_tiles, &hl->total_chunks, d, tile_keys);
    }
}

}  // namespace

size_t bucket_workspace_bytes(int key_bytes, bool vals, size_t n, size_t nb) {
    if (nb == 0) nb = std::max<size_t>(1, n / 16);
    return bucket_layout(plan_info(key_bytes, vals, n, nb, false, 0, 0)).total;
}

template <typename KeyT, bool VALS>
static rs_status bucket_sort_t(const KeyT* keys_in, KeyT* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                               size_t n, uint64_t min_key, uint64_t max_key, size_t nb, void* ws, size_t ws_bytes,
                               cudaStream_t stream) {
    const bool bounds_known = min_key <= max_key;
    const BucketPlanInfo I = plan_info(sizeof(KeyT), VALS, n, nb, bounds_known, min_key, max_key);
    const BucketLayout L = bucket_layout(I);
    if (ws_bytes < L.total) return RS_ERR_WORKSPACE;
    unsigned char* base = static_cast<unsigned char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
    BucketParams* bp = reinterpret_cast<BucketParams*>(base + L.off_params);
    unsigned long long* mm = reinterpret_cast<unsigned long long*>(base + L.off_mm);
    SegPlanHdr* h = reinterpret_cast<SegPlanHdr*>(base + L.off_hdr);
    SegPlanHdr* h_leaf1 = h + 0;  // num_small: leaf1 count, num_next: copy count
    SegPlanHdr* h_next = h + 1;   // level-2 parents (num_large, tiles, chunks), num_small: leaf2 count
    SegPlanHdr* h_ovf = h + 2;    // overflow partitions
    uint32_t* counts1 = reinterpret_cast<uint32_t*>(base + L.off_counts1);
    uint32_t* scan1 = reinterpret_cast<uint32_t*>(base + L.off_scan1);
    SegDesc* leaf1 = reinterpret_cast<SegDesc*>(base + L.off_leaf1);
    SegDesc* copyl = reinterpret_cast<SegDesc*>(base + L.off_copy);
    SegDesc* next = reinterpret_cast<SegDesc*>(base + L.off_next);
    SegDesc* leaf2 = reinterpret_cast<SegDesc*>(base + L.off_leaf2);
    SegDesc* ovf = reinterpret_cast<SegDesc*>(base + L.off_ovf);
    uint32_t* tile_seg = reinterpret_cast<uint32_t*>(base + L.off_tile_seg);
    uint32_t* chunk_seg = reinterpret_cast<uint32_t*>(base + L.off_chunk_seg);
    uint32_t* rows = reinterpret_cast<uint32_t*>(base + L.off_rows);
    uint32_t* status[2] = {reinterpret_cast<uint32_t*>(base + L.off_status0),
                           reinterpret_cast<uint32_t*>(base + L.off_status1)};
    KeyT* tmp_k = reinterpret_cast<KeyT*>(base + L.off_tmp_keys);
    uint32_t* tmp_v = VALS ? reinterpret_cast<uint32_t*>(base + L.off_tmp_vals) : nullptr;
    const uint32_t tk = BucketShape<KeyT, VALS>::kTile;

    // header, plan counters and level-1 counts start at zero
    RS_CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(h, 0, 4 * sizeof(SegPlanHdr), stream));
    RS_CUDA_TRY(cudaMemsetAsync(counts1, 0, 256 * 4, stream));

    // b1: bounds (Algorithm 2 assumes every key lies in [min, max])
    if (!bounds_known) {
        RS_CUDA_TRY(cudaMemsetAsync(mm, 0xff, 8, stream));
        RS_CUDA_TRY(cudaMemsetAsync(mm + 1, 0, 8, stream));
        KernelScope scope("minmax", stream);
        size_t grid = std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 8);
        k_minmax<KeyT><<<(unsigned)std::max<size_t>(grid, 1), 256, 0, stream>>>(keys_in, n, mm);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    {
        KernelScope scope("bucket_params", stream);
        k_bucket_params<<<1, 32, 0, stream>>>(bp, bounds_known ? nullptr : mm, min_key, max_key, nb, (int)sizeof(KeyT));
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }

    // b2-b4, level 1: count the top digit of every bucket id, prefix, stable scatter keys_in -> buffer
    const uint32_t bins1 = 1u << I.d1;
    const uint32_t tiles1 = (uint32_t)((n + tk - 1) / tk);
    {
        CountParams cp{};
        cp.keys = keys_in;
        cp.n = n;
        cp.passes = 1;
        cp.bins = bins1;
        cp.counts = counts1;
        cp.scan = scan1;
        cp.zero_ptr = status[0];
        cp.zero_words = (size_t)tiles1 * bins1;
        cp.hdr = hdr;
        BucketCountDigits dg{bp, I.shift1, bins1 - 1u, {}};
        if (launch_counts<KeyT>(cp, dg, count_grid(n), stream) != cudaSuccess) return RS_ERR_CUDA;
    }
    {
        PassParams<BucketDigit> pp{};
        pp.keys_in = keys_in;
        pp.keys_out = tmp_k;
        pp.vals_in = vals_in;
        pp.vals_out = tmp_v;
        pp.n = (uint32_t)n;
        pp.num_tiles = tiles1;
        pp.digit_bits = I.d1;
        pp.op = BucketDigit{bp, I.shift1, bins1 - 1u, {}};
        pp.digit_base = scan1;
        pp.status = status[0];
        pp.status_next = status[1];
        pp.tile_ctr = &hdr->tile_ctr[0];
        pp.hdr = hdr;
        pp.spin_limit = debug_spin_limit();
        pp.stall_tile = debug_stall_tile();
        if (launch_plain_bucket_pass<KeyT, VALS>(pp, stream) != cudaSuccess) return RS_ERR_CUDA;
    }
    PlanLevel pl{};
    pl.bp = bp;
    pl.cap = kLocalCap;
    pl.tile_keys = tk;
    pl.ovf_tile_keys = SegShape<KeyT, VALS>::kTile;  // the overflow passes run the segmented radix shape
    pl.key_width = 8 * (int)sizeof(KeyT);
    pl.copy = copyl;
    pl.num_copy = &h_leaf1->num_next;
    pl.ovf = ovf;
    pl.ovf_hdr = h_ovf;
    {
        pl.shift = I.shift1;
        pl.digit_bits = I.d1;
        pl.parents = nullptr;
        pl.n_total = n;
        pl.starts = scan1;
        pl.counts = counts1;
        pl.in_out = 0;
        pl.leaf = leaf1;
        pl.num_leaf = &h_leaf1->num_small;
        pl.next = I.level2 ? next : nullptr;
        pl.next_hdr = h_next;
        KernelScope scope("bucket_plan", stream);
        k_bucket_plan<<<1, 256, 0, stream>>>(pl);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }

    // level 2: partitions above the shared-memory capacity, by the next digit, buffer -> keys_out
    if (I.level2) {
        const uint32_t bins2 = 1u << I.d2;
        const size_t parents2 = bins1;
        {
            KernelScope scope("plan_maps", stream);
            k_plan_maps<<<(unsigned)std::min<size_t>(parents2, (size_t)device_sm_count() * 2), 256, 0, stream>>>(
                next, h_next, tk, tile_seg, chunk_seg);
            if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
        }
        RS_CUDA_TRY(cudaMemsetAsync(rows, 0, parents2 * bins2 * 4, stream));
        BucketDigits dg{bp, I.shift2, bins2 - 1u, {}};
        if (launch_seg_counts<KeyT>(tmp_k, next, h_next, chunk_seg, I.max_chunks, dg, 1, bins2, rows, status[0],
                                    I.max_tiles * (size_t)bins2, stream) != cudaSuccess)
            return RS_ERR_CUDA;
        {
            KernelScope scope("seg_scan", stream);
            k_seg_scan<<<(unsigned)std::min<size_t>(parents2, (size_t)device_sm_count() * 2), 256,
                         (bins2 + 256 / 32 + 1) * 4, stream>>>(rows, h_next, 1, bins2, 0);
            if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
        }
        SegPassParams<BucketDigit> sp{};
        sp.base.keys_in = tmp_k;
        sp.base.keys_out = keys_out;
        sp.base.vals_in = tmp_v;
        sp.base.vals_out = vals_out;
        sp.base.digit_bits = I.d2;
        sp.base.op = BucketDigit{bp, I.shift2, bins2 - 1u, {}};
        sp.base.status = status[0];
        sp.base.status_next = nullptr;
        sp.base.tile_ctr = &hdr->tile_ctr[1];
        sp.base.hdr = hdr;
        sp.base.spin_limit = debug_spin_limit();
        sp.base.stall_tile = debug_stall_tile();
        sp.segs = next;
        sp.hdr = h_next;
        sp.tile_seg = tile_seg;
        sp.seg_base = rows;
        sp.pass = 0;
        sp.passes = 1;
        if (launch_bucket_seg_pass<KeyT, VALS, BucketDigit>(sp, I.max_tiles, stream) != cudaSuccess) return RS_ERR_CUDA;
        pl.shift = I.shift2;
        pl.digit_bits = I.d2;
        pl.parents = next;
        pl.num_parents = &h_next->num_large;
        pl.starts = rows;
        pl.counts = nullptr;
        pl.in_out = 1;
        pl.leaf = leaf2;
        pl.num_leaf = &h_next->num_small;
        pl.next = nullptr;
        KernelScope scope("bucket_plan", stream);
        k_bucket_plan<<<(unsigned)parents2, 256, 0, stream>>>(pl);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }

    // partitions that can hold only one key value move unchanged
    {
        KernelScope scope("copy_segments", stream);
        k_copy_segments<KeyT><<<bins1, 256, 0, stream>>>(tmp_k, tmp_v, keys_out, vals_out, copyl, &h_leaf1->num_next);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // b5: sort each bucket of the shared-memory partitions
    rs_status st = enqueue_local_sorts(sizeof(KeyT), VALS, tmp_k, tmp_v, keys_out, vals_out, leaf1,
                                       &h_leaf1->num_small, bins1, bp, nullptr, stream);
    if (st != RS_OK) return st;
    if (I.level2) {
        st = enqueue_local_sorts(sizeof(KeyT), VALS, keys_out, vals_out, keys_out, vals_out, leaf2,
                                 &h_next->num_small, I.max_leaf2, bp, nullptr, stream);
        if (st != RS_OK) return st;
    }
    // overflow partitions: radix on the key bits their buckets span
    if (I.ovf_passes > 0) {
        SegBuffers B{};
        B.ws_hdr = hdr;
        B.hdr = h_ovf;
        B.large = ovf;
        B.small = nullptr;
        B.tile_seg = tile_seg;
        B.chunk_seg = chunk_seg;
        B.seg_rows = rows;
        B.status[0] = status[0];
        B.status[1] = status[1];
        B.tmp_keys = tmp_k;
        B.tmp_vals = tmp_v;
        B.max_segs = I.max_ovf;
        B.max_tiles = I.max_tiles;
        B.max_chunks = I.max_chunks;
        B.max_passes = I.ovf_passes;
        B.max_bins = 256;
        const void* src_k = I.level2 ? static_cast<const void*>(keys_out) : static_cast<const void*>(tmp_k);
        const uint32_t* src_v = VALS ? (I.level2 ? vals_out : tmp_v) : nullptr;
        // the tile counters of these passes follow the two used above
        B.ws_hdr = hdr;
        st = enqueue_large_passes_at(sizeof(KeyT), VALS, src_k, src_v, keys_out, vals_out, B, I.ovf_passes,
                                     I.ovf_bits, 2, stream);
        if (st != RS_OK) return st;
    }
    return RS_OK;
}

static rs_status bucket_impl_body(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                  uint32_t* vals_out, size_t n, uint64_t min_key, uint64_t max_key, size_t nb,
                                  void* ws, size_t ws_bytes, cudaStream_t stream);

static rs_status bucket_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                             uint32_t* vals_out, size_t n, uint64_t min_key, uint64_t max_key, size_t nb, void* ws,
                             size_t ws_bytes, cudaStream_t stream) {
    NvtxRange range(key_bytes == 4 ? "bs_sort_u32" : "bs_sort_u64");
    rs_status st = bucket_impl_body(key_bytes, keys_in, keys_out, vals_in, vals_out, n, min_key, max_key, nb, ws,
                                    ws_bytes, stream);
    if (st == RS_OK && n > 1 && checked_mode())
        st = enqueue_order_check(key_bytes, keys_out, n, KeyXform{}, static_cast<WsHeader*>(ws), stream);
    return st;
}

static rs_status bucket_impl_body(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                  uint32_t* vals_out, size_t n, uint64_t min_key, uint64_t max_key, size_t nb,
                                  void* ws, size_t ws_bytes, cudaStream_t stream) {
    if ((vals_in == nullptr) != (vals_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS) return RS_ERR_INVALID_ARG;
    if (n == 0) return RS_OK;
    if (!keys_in || !keys_out) return RS_ERR_INVALID_ARG;
    if (nb == 0) nb = std::max<size_t>(1, n / 16);
    if (nb > ((size_t)1 << 32)) return RS_ERR_INVALID_ARG;
    const bool vals = vals_in != nullptr;
    const size_t kb = n * key_bytes, vb = n * 4;
    if (keys_in != keys_out && ranges_overlap(keys_in, kb, keys_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && vals_in != vals_out && ranges_overlap(vals_in, vb, vals_out, vb)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)keys_in | (uintptr_t)keys_out) % key_bytes) return RS_ERR_INVALID_ARG;
    if (vals && (((uintptr_t)vals_in | (uintptr_t)vals_out) % 4)) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    if (key_bytes == 4)
        return vals ? bucket_sort_t<uint32_t, true>(static_cast<const uint32_t*>(keys_in),
                                                    static_cast<uint32_t*>(keys_out), vals_in, vals_out, n, min_key,
                                                    max_key, nb, ws, ws_bytes, stream)
                    : bucket_sort_t<uint32_t, false>(static_cast<const uint32_t*>(keys_in),
                                                     static_cast<uint32_t*>(keys_out), vals_in, vals_out, n, min_key,
                                                     max_key, nb, ws, ws_bytes, stream);
    return vals ? bucket_sort_t<uint64_t, true>(static_cast<const uint64_t*>(keys_in), static_cast<uint64_t*>(keys_out),
                                                vals_in, vals_out, n, min_key, max_key, nb, ws, ws_bytes, stream)
                : bucket_sort_t<uint64_t, false>(static_cast<const uint64_t*>(keys_in),
                                                 static_cast<uint64_t*>(keys_out), vals_in, vals_out, n, min_key,
                                                 max_key, nb, ws, ws_bytes, stream);
}

static rs_status bucket_counts_impl(int key_bytes, const void* keys, size_t n, uint64_t min_key, uint64_t max_key,
                                    size_t nb, uint32_t* counts, void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (min_key > max_key || nb == 0 || nb > ((size_t)1 << 32) || !counts || ((uintptr_t)counts % 4))
        return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS || (n && !keys) || ((uintptr_t)keys % key_bytes)) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    if (ws_bytes < 512 + sizeof(BucketParams)) return RS_ERR_WORKSPACE;
    unsigned char* base = static_cast<unsigned char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
    BucketParams* bp = reinterpret_cast<BucketParams*>(base + 256);
    RS_CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(counts, 0, nb * 4, stream));
    {
        KernelScope scope("bucket_params", stream);
        k_bucket_params<<<1, 32, 0, stream>>>(bp, nullptr, min_key, max_key, nb, key_bytes);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    if (n == 0) return RS_OK;
    const size_t grid = std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 8);
    KernelScope scope("bucket_counts", stream);
    if (key_bytes == 4)
        k_bucket_counts<uint32_t><<<(unsigned)grid, 256, 0, stream>>>(static_cast<const uint32_t*>(keys), n, bp,
                                                                     counts, hdr);
    else
        k_bucket_counts<uint64_t><<<(unsigned)grid, 256, 0, stream>>>(static_cast<const uint64_t*>(keys), n, bp,
                                                                     counts, hdr);
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}


// ---------------------------------------------------------------- segmented bucket sort: host
namespace {

struct SegBucketLayout {
    size_t max_large, max_runs1, max_next, max_runs2, max_ovf, max_tiles, max_chunks, max_rows;
    int ovf_passes, ovf_bits;
    size_t off_table, off_mm, off_hdr, off_all, off_small, off_large, off_leaf1, off_copy, off_next, off_leaf2,
        off_ovf, off_tile_seg, off_chunk_seg, off_rows, off_status0, off_status1, off_tmp_keys, off_tmp_vals, total;
};

int floor_log2_host(uint64_t x) { return x ? bit_length_host(x) - 1 : 0; }

// Sizes of every list and buffer for nseg segments over n_total keys.  The
// bounds: a large segment, a level-1 child sent to level 2 and an overflow
// partition each hold more than kLocalCap keys; every leaf run holds a key
// and lies in one large segment, whose level has at most 256 children.
// Overflow partitions span at most 2^shift2 buckets of a segment with at
// least (kLocalCap + 1) / keys_per_bucket buckets, so their keys span at most
// range / min(2^15, that) + 2 values (range: the declared one, else 2^width);
// the overflow radix passes cover that many bits, in an even number of
// passes because their input and output are keys_out.
SegBucketLayout seg_bucket_layout(int key_bytes, bool vals, size_t n_total, size_t nseg, uint64_t keys_per_bucket,
                                  bool bounds_known, uint64_t min_key, uint64_t max_key) {
    SegBucketLayout L{};
    const size_t big = n_total / (kLocalCap + 1) + 1;
    const uint32_t tk = std::min(seg_tile_keys(key_bytes, vals), bucket_tile_keys(key_bytes, vals));
    L.max_large = std::min<size_t>(std::max<size_t>(nseg, 1), big);
    L.max_runs1 = std::min<size_t>(256 * L.max_large, n_total + 1);
    L.max_next = big;
    L.max_runs2 = std::min<size_t>(256 * L.max_next, n_total + 1);
    L.max_ovf = big;
    const size_t most_lists = std::max(L.max_large, L.max_next);
    L.max_tiles = n_total / tk + most_lists + 2;
    L.max_chunks = n_total / kSegChunk + std::max<size_t>(std::max<size_t>(nseg, 1), most_lists) + 2;
    const int width = 8 * key_bytes;
    const int range_bits = bounds_known ? (max_key - min_key == ~0ull ? 64 : bit_length_host(max_key - min_key)) : width;
    const uint64_t nb_min = std::max<uint64_t>(1, (kLocalCap + 1) / keys_per_bucket);
    int bits = range_bits - std::min(15, floor_log2_host(nb_min)) + 2;
    bits = std::max(1, std::min(width, bits));
    int P = (bits + 7) / 8;
    if (P % 2) ++P;
    L.ovf_passes = P;
    L.ovf_bits = (bits + P - 1) / P;
    L.max_rows = std::max<size_t>(most_lists * 256, L.max_ovf * (size_t)P * 256);
    Carver c;
    c.take(sizeof(WsHeader));
    L.off_table = c.take(std::max<size_t>(nseg, 1) * sizeof(BucketParams));
    L.off_mm = c.take(std::max<size_t>(nseg, 1) * 16);
    L.off_hdr = c.take(5 * sizeof(SegPlanHdr));
    L.off_all = c.take(std::max<size_t>(nseg, 1) * sizeof(SegDesc));
    L.off_small = c.take(std::max<size_t>(nseg, 1) * sizeof(SegDesc));
    L.off_large = c.take(L.max_large * sizeof(SegDesc));
    L.off_leaf1 = c.take(L.max_runs1 * sizeof(SegDesc));
    L.off_copy = c.take(L.max_runs1 * sizeof(SegDesc));
    L.off_next = c.take(L.max_next * sizeof(SegDesc));
    L.off_leaf2 = c.take(L.max_runs2 * sizeof(SegDesc));
    L.off_ovf = c.take(L.max_ovf * sizeof(SegDesc));
    L.off_tile_seg = c.take(L.max_tiles * 4);
    L.off_chunk_seg = c.take(L.max_chunks * 4);
    L.off_rows = c.take(L.max_rows * 4);
    L.off_status0 = c.take(L.max_tiles * 256 * 4);
    L.off_status1 = c.take(L.max_tiles * 256 * 4);
    L.off_tmp_keys = c.take(n_total * key_bytes);
    L.off_tmp_vals = vals ? c.take(n_total * 4) : 0;
    L.total = c.off;
    return L;
}

}  // namespace

size_t seg_bucket_workspace_bytes(int key_bytes, bool vals, size_t n_total, size_t nseg, size_t keys_per_bucket) {
    if (keys_per_bucket == 0) keys_per_bucket = 16;
    // the bound with unknown bounds covers every declared range
    return seg_bucket_layout(key_bytes, vals, n_total, nseg, keys_per_bucket, false, 0, 0).total;
}

template <typename KeyT, bool VALS>
static rs_status seg_bucket_sort_t(const KeyT* keys_in, KeyT* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                                   const uint64_t* d_offsets, size_t nseg, size_t n_total, uint64_t min_key,
                                   uint64_t max_key, uint64_t kpb, void* ws, size_t ws_bytes, cudaStream_t stream) {
    const bool bounds_known = min_key <= max_key;
    const SegBucketLayout L = seg_bucket_layout(sizeof(KeyT), VALS, n_total, nseg, kpb, bounds_known, min_key, max_key);
    if (ws_bytes < L.total) return RS_ERR_WORKSPACE;
    unsigned char* base = static_cast<unsigned char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
    BucketParams* table = reinterpret_cast<BucketParams*>(base + L.off_table);
    unsigned long long* mm = bounds_known ? nullptr : reinterpret_cast<unsigned long long*>(base + L.off_mm);
    SegPlanHdr* h = reinterpret_cast<SegPlanHdr*>(base + L.off_hdr);
    SegPlanHdr* h_all = h + 0;    // listed segments (min/max chunks)
    SegPlanHdr* h_seg = h + 1;    // num_small: whole small segments; num_large, tiles, chunks: level-1 parents
    SegPlanHdr* h_leaf1 = h + 2;  // num_small: level-1 leaf runs, num_next: copies
    SegPlanHdr* h_next = h + 3;   // level-2 parents (num_large, tiles, chunks), num_small: level-2 leaf runs
    SegPlanHdr* h_ovf = h + 4;    // overflow partitions
    auto desc = [&](size_t off) { return reinterpret_cast<SegDesc*>(base + off); };
    SegDesc *all = desc(L.off_all), *small = desc(L.off_small), *large = desc(L.off_large);
    SegDesc *leaf1 = desc(L.off_leaf1), *copyl = desc(L.off_copy), *next = desc(L.off_next);
    SegDesc *leaf2 = desc(L.off_leaf2), *ovf = desc(L.off_ovf);
    uint32_t* tile_seg = reinterpret_cast<uint32_t*>(base + L.off_tile_seg);
    uint32_t* chunk_seg = reinterpret_cast<uint32_t*>(base + L.off_chunk_seg);
    uint32_t* rows = reinterpret_cast<uint32_t*>(base + L.off_rows);
    uint32_t* status[2] = {reinterpret_cast<uint32_t*>(base + L.off_status0),
                           reinterpret_cast<uint32_t*>(base + L.off_status1)};
    KeyT* tmp_k = reinterpret_cast<KeyT*>(base + L.off_tmp_keys);
    uint32_t* tmp_v = VALS ? reinterpret_cast<uint32_t*>(base + L.off_tmp_vals) : nullptr;
    const uint32_t tk = BucketShape<KeyT, VALS>::kTile;
    const int sms = device_sm_count();
    const unsigned seg_grid = (unsigned)((nseg + 255) / 256);
    const int check = bounds_known ? 1 : 0;

    RS_CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(h, 0, 5 * sizeof(SegPlanHdr), stream));
    // b1 per segment: the offsets are checked, and without declared bounds
    // each segment's min and max are reduced
    {
        KernelScope scope("segb_list", stream);
        k_segb_list<<<seg_grid, 256, 0, stream>>>(d_offsets, nseg, n_total, all, h_all, mm, hdr);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    if (!bounds_known) {
        {
            KernelScope scope("segb_chunk_map", stream);
            k_segb_chunk_map<<<(unsigned)std::min<size_t>(nseg, (size_t)sms * 8), 256, 0, stream>>>(all, h_all,
                                                                                                    chunk_seg);
            if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
        }
        KernelScope scope("minmax", stream);
        k_segb_minmax<KeyT><<<(unsigned)std::min<size_t>(L.max_chunks, (size_t)sms * 8), 256, 0, stream>>>(
            keys_in, all, h_all, chunk_seg, mm);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    {
        KernelScope scope("segb_classify", stream);
        k_segb_classify<<<seg_grid, 256, 0, stream>>>(d_offsets, nseg, n_total, mm, min_key, max_key, kpb,
                                                      (int)sizeof(KeyT), tk, table, small, large, h_seg);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // level 1 over the large segments: counts of each segment's top bucket-id
    // digit, prefixes, stable partition keys_in -> buffer, plan
    const unsigned big_grid = (unsigned)std::min<size_t>(L.max_large, (size_t)sms * 8);
    {
        KernelScope scope("plan_maps", stream);
        k_plan_maps<<<big_grid, 256, 0, stream>>>(large, h_seg, tk, tile_seg, chunk_seg);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    RS_CUDA_TRY(cudaMemsetAsync(rows, 0, L.max_large * 256 * 4, stream));
    {
        BucketDigits dg{nullptr, 0, 0u, {}, table, 1, check};
        if (launch_seg_counts<KeyT>(keys_in, large, h_seg, chunk_seg, L.max_chunks, dg, 1, 256, rows, status[0],
                                    L.max_tiles * 256, stream, hdr) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    {
        KernelScope scope("seg_scan", stream);
        k_seg_scan<<<big_grid, 256, (256 + 256 / 32 + 1) * 4, stream>>>(rows, h_seg, 1, 256, 0);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    SegPassParams<BucketDigit> sp{};
    sp.base.digit_bits = 8;
    sp.base.hdr = hdr;
    sp.base.spin_limit = debug_spin_limit();
    sp.base.stall_tile = debug_stall_tile();
    sp.tile_seg = tile_seg;
    sp.seg_base = rows;
    sp.pass = 0;
    sp.passes = 1;
    sp.base.keys_in = keys_in;
    sp.base.keys_out = tmp_k;
    sp.base.vals_in = vals_in;
    sp.base.vals_out = tmp_v;
    sp.base.op = BucketDigit{nullptr, 0, 0u, {}, table, 1};
    sp.base.status = status[0];
    sp.base.status_next = nullptr;
    sp.base.tile_ctr = &hdr->tile_ctr[0];
    sp.segs = large;
    sp.hdr = h_seg;
    if (launch_bucket_seg_pass<KeyT, VALS, BucketDigit>(sp, L.max_tiles, stream) != cudaSuccess) return RS_ERR_CUDA;
    PlanLevel pl{};
    pl.table = table;
    pl.row_stride = 256;
    pl.cap = kLocalCap;
    pl.tile_keys = tk;
    pl.ovf_tile_keys = SegShape<KeyT, VALS>::kTile;  // the overflow passes run the segmented radix shape
    pl.key_width = 8 * (int)sizeof(KeyT);
    pl.copy = copyl;
    pl.num_copy = &h_leaf1->num_next;
    pl.ovf = ovf;
    pl.ovf_hdr = h_ovf;
    {
        pl.level = 1;
        pl.parents = large;
        pl.num_parents = &h_seg->num_large;
        pl.starts = rows;
        pl.in_out = 0;
        pl.leaf = leaf1;
        pl.num_leaf = &h_leaf1->num_small;
        pl.next = next;
        pl.next_hdr = h_next;
        KernelScope scope("bucket_plan", stream);
        k_bucket_plan<<<big_grid, 256, 0, stream>>>(pl);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // level 2 over the children still above kLocalCap keys: next digit,
    // buffer -> keys_out, plan (big children left go to the overflow radix)
    const unsigned next_grid = (unsigned)std::min<size_t>(L.max_next, (size_t)sms * 8);
    {
        KernelScope scope("plan_maps", stream);
        k_plan_maps<<<next_grid, 256, 0, stream>>>(next, h_next, tk, tile_seg, chunk_seg);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    RS_CUDA_TRY(cudaMemsetAsync(rows, 0, L.max_next * 256 * 4, stream));
    {
        BucketDigits dg{nullptr, 0, 0u, {}, table, 2, 0};
        if (launch_seg_counts<KeyT>(tmp_k, next, h_next, chunk_seg, L.max_chunks, dg, 1, 256, rows, status[0],
                                    L.max_tiles * 256, stream) != cudaSuccess)
            return RS_ERR_CUDA;
    }
    {
        KernelScope scope("seg_scan", stream);
        k_seg_scan<<<next_grid, 256, (256 + 256 / 32 + 1) * 4, stream>>>(rows, h_next, 1, 256, 0);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    sp.base.keys_in = tmp_k;
    sp.base.keys_out = keys_out;
    sp.base.vals_in = tmp_v;
    sp.base.vals_out = vals_out;
    sp.base.op = BucketDigit{nullptr, 0, 0u, {}, table, 2};
    sp.base.tile_ctr = &hdr->tile_ctr[1];
    sp.segs = next;
    sp.hdr = h_next;
    if (launch_bucket_seg_pass<KeyT, VALS, BucketDigit>(sp, L.max_tiles, stream) != cudaSuccess) return RS_ERR_CUDA;
    {
        pl.level = 2;
        pl.parents = next;
        pl.num_parents = &h_next->num_large;
        pl.starts = rows;
        pl.in_out = 1;
        pl.leaf = leaf2;
        pl.num_leaf = &h_next->num_small;
        pl.next = nullptr;
        KernelScope scope("bucket_plan", stream);
        k_bucket_plan<<<next_grid, 256, 0, stream>>>(pl);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // level-1 partitions that can hold only one key value move unchanged
    {
        KernelScope scope("copy_segments", stream);
        k_copy_segments<KeyT><<<(unsigned)std::min<size_t>(L.max_runs1, (size_t)sms * 8), 256, 0, stream>>>(
            tmp_k, tmp_v, keys_out, vals_out, copyl, &h_leaf1->num_next);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // b5: every bucket of the leaf runs (level 1 from the buffer, level 2 in
    // place), and every small segment whole, from keys_in (it reads its
    // whole segment before writing, so keys_in == keys_out is fine)
    rs_status st = enqueue_local_sorts(sizeof(KeyT), VALS, tmp_k, tmp_v, keys_out, vals_out, leaf1,
                                       &h_leaf1->num_small, L.max_runs1, nullptr, nullptr, stream, table, 0);
    if (st != RS_OK) return st;
    st = enqueue_local_sorts(sizeof(KeyT), VALS, keys_out, vals_out, keys_out, vals_out, leaf2, &h_next->num_small,
                             L.max_runs2, nullptr, nullptr, stream, table, 0);
    if (st != RS_OK) return st;
    st = enqueue_local_sorts(sizeof(KeyT), VALS, keys_in, vals_in, keys_out, vals_out, small, &h_seg->num_small,
                             nseg, nullptr, hdr, stream, table, check);
    if (st != RS_OK) return st;
    // overflow partitions: radix on the key bits their buckets span, keys_out -> keys_out
    SegBuffers B{};
    B.ws_hdr = hdr;
    B.hdr = h_ovf;
    B.large = ovf;
    B.tile_seg = tile_seg;
    B.chunk_seg = chunk_seg;
    B.seg_rows = rows;
    B.status[0] = status[0];
    B.status[1] = status[1];
    B.tmp_keys = tmp_k;
    B.tmp_vals = tmp_v;
    B.max_segs = L.max_ovf;
    B.max_tiles = L.max_tiles;
    B.max_chunks = L.max_chunks;
    B.max_passes = L.ovf_passes;
    B.max_bins = 256;
    return enqueue_large_passes_at(sizeof(KeyT), VALS, keys_out, vals_out, keys_out, vals_out, B, L.ovf_passes,
                                   L.ovf_bits, 2, stream);
}

static rs_status seg_bucket_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                 uint32_t* vals_out, const uint64_t* d_offsets, size_t nseg, size_t n_total,
                                 uint64_t min_key, uint64_t max_key, size_t kpb, void* ws, size_t ws_bytes,
                                 cudaStream_t stream) {
    if ((vals_in == nullptr) != (vals_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (kpb == 0) kpb = 16;
    if (kpb > ((size_t)1 << 30)) return RS_ERR_INVALID_ARG;
    const bool vals = vals_in != nullptr;
    if (nseg == 0 || n_total == 0) return RS_OK;
    if (!d_offsets || !keys_in || !keys_out) return RS_ERR_INVALID_ARG;
    if (nseg > ((size_t)1 << 31)) return RS_ERR_INVALID_ARG;
    const size_t kb = n_total * key_bytes, vb = n_total * 4;
    if (keys_in != keys_out && ranges_overlap(keys_in, kb, keys_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && vals_in != vals_out && ranges_overlap(vals_in, vb, vals_out, vb)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)keys_in | (uintptr_t)keys_out) % key_bytes) return RS_ERR_INVALID_ARG;
    if (vals && (((uintptr_t)vals_in | (uintptr_t)vals_out) % 4)) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    if (key_bytes == 4) {
        if (min_key <= max_key && max_key > 0xffffffffull) return RS_ERR_INVALID_ARG;
        return vals ? seg_bucket_sort_t<uint32_t, true>(static_cast<const uint32_t*>(keys_in),
                                                        static_cast<uint32_t*>(keys_out), vals_in, vals_out, d_offsets,
                                                        nseg, n_total, min_key, max_key, kpb, ws, ws_bytes, stream)
                    : seg_bucket_sort_t<uint32_t, false>(static_cast<const uint32_t*>(keys_in),
                                                         static_cast<uint32_t*>(keys_out), vals_in, vals_out,
                                                         d_offsets, nseg, n_total, min_key, max_key, kpb, ws,
                                                         ws_bytes, stream);
    }
    return vals ? seg_bucket_sort_t<uint64_t, true>(static_cast<const uint64_t*>(keys_in),
                                                    static_cast<uint64_t*>(keys_out), vals_in, vals_out, d_offsets,
                                                    nseg, n_total, min_key, max_key, kpb, ws, ws_bytes, stream)
                : seg_bucket_sort_t<uint64_t, false>(static_cast<const uint64_t*>(keys_in),
                                                     static_cast<uint64_t*>(keys_out), vals_in, vals_out, d_offsets,
                                                     nseg, n_total, min_key, max_key, kpb, ws, ws_bytes, stream);
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status bs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      size_t n, uint32_t min_key, uint32_t max_key, size_t num_buckets, void* ws, size_t ws_bytes,
                      rs_stream_t stream) {
    return bucket_impl(4, keys_in, keys_out, vals_in, vals_out, n, min_key, max_key, num_buckets, ws, ws_bytes,
                       stream);
}

rs_status bs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      size_t n, uint64_t min_key, uint64_t max_key, size_t num_buckets, void* ws, size_t ws_bytes,
                      rs_stream_t stream) {
    return bucket_impl(8, keys_in, keys_out, vals_in, vals_out, n, min_key, max_key, num_buckets, ws, ws_bytes,
                       stream);
}

size_t bs_segmented_workspace_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg,
                                    size_t keys_per_bucket) {
    if (key_bytes != 4 && key_bytes != 8) return 0;
    return seg_bucket_workspace_bytes(key_bytes, has_values != 0, n_total, nseg, keys_per_bucket);
}

rs_status bs_sort_segmented_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                uint32_t min_key, uint32_t max_key, size_t keys_per_bucket, void* ws, size_t ws_bytes,
                                rs_stream_t stream) {
    return seg_bucket_impl(4, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, min_key, max_key,
                           keys_per_bucket, ws, ws_bytes, stream);
}

rs_status bs_sort_segmented_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                uint64_t min_key, uint64_t max_key, size_t keys_per_bucket, void* ws, size_t ws_bytes,
                                rs_stream_t stream) {
    return seg_bucket_impl(8, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, min_key, max_key,
                           keys_per_bucket, ws, ws_bytes, stream);
}

rs_status bs_bucket_counts_u32(const uint32_t* keys, size_t n, uint32_t min_key, uint32_t max_key, size_t num_buckets,
                               uint32_t* d_counts, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return bucket_counts_impl(4, keys, n, min_key, max_key, num_buckets, d_counts, ws, ws_bytes, stream);
}

rs_status bs_bucket_counts_u64(const uint64_t* keys, size_t n, uint64_t min_key, uint64_t max_key, size_t num_buckets,
                               uint32_t* d_counts, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return bucket_counts_impl(8, keys, n, min_key, max_key, num_buckets, d_counts, ws, ws_bytes, stream);
}

}  // extern "C"
