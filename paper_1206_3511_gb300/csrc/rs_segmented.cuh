// rs_segmented.cuh -- kernels that sort many independent segments of one
// array: device-side planning, per-segment digit counts, a segmented
// one-sweep scatter pass and a shared-memory sort for segments that fit in
// one block.  Each segment is sorted exactly as Algorithm 4 (Sec. 2.5) would
// sort it alone.  The bucket sort reuses these kernels for its partitions.
#pragma once

#include "rs_onesweep.cuh"

namespace rs {

// One segment of the arrays.  Keys are sorted on the low `bits` bits of
// (key - key_lo).
struct SegDesc {
    uint64_t start;   // index of the segment's first key
    uint64_t key_lo;  // subtracted from every key before digits are taken
    uint32_t n;       // number of keys
    uint32_t tile0;   // first global tile (scatter passes)
    uint32_t chunk0;  // first counting chunk
    uint32_t bits;    // key bits to sort on
    uint64_t aux;     // planner data (bucket range of bucket-sort partitions)
    uint32_t grp;     // input segment the descriptor belongs to (segmented bucket sort: its bucket parameters)
    uint32_t pad;
};
static_assert(sizeof(SegDesc) == 48, "SegDesc layout");

// Device-side totals of a plan (zeroed before planning).
struct SegPlanHdr {
    uint32_t num_large;     // segments sorted by scatter passes
    uint32_t num_small;     // segments sorted in shared memory
    uint32_t total_tiles;   // scatter-pass tiles over all large segments
    uint32_t total_chunks;  // counting chunks over all large segments
    uint32_t num_next;      // partitions handed to the next level (bucket sort)
    uint32_t next_tiles;
    uint32_t next_chunks;
    uint32_t num_tiny;      // segments sorted by one warp each
};

constexpr uint32_t kSegChunk = 32768;  // keys per counting block

__device__ __forceinline__ uint32_t ceil_div_u32(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

// Append one segment to a list with its tile and chunk ranges reserved.
__device__ __forceinline__ void append_large(SegDesc* list, uint32_t* count, uint32_t* tiles, uint32_t* chunks,
                                             SegDesc d, uint32_t tile_keys) {
    d.tile0 = atomicAdd(tiles, ceil_div_u32(d.n, tile_keys));
    d.chunk0 = atomicAdd(chunks, ceil_div_u32(d.n, kSegChunk));
    list[atomicAdd(count, 1u)] = d;
}

// Segments of at most this many keys are sorted by one warp each.
constexpr uint32_t kTinyCap = 256;

// Segments from an offset table: empty ones are dropped, those of at most
// kTinyCap keys go to the warp list (when `tiny` is given), those of at most
// `small_cap` keys to the shared-memory list, the others to the scatter
// list.  One thread per segment.  A segment whose offsets decrease, that ends
// past n_total keys, or that is above the single-sort limit is dropped and
// reported as RS_ERR_INVALID_ARG: every segment kept lies inside the arrays,
// so the tiles and chunks reserved for them stay within the workspace's
// bounds (at most n_total / tile + nseg + 1 tiles).
static __global__ void k_plan_from_offsets(const uint64_t* __restrict__ offsets, size_t nseg, uint64_t n_total,
                                           uint32_t small_cap, uint32_t tile_keys, int bits, SegDesc* large,
                                           SegDesc* small, SegDesc* tiny, SegPlanHdr* hdr, WsHeader* ws_hdr) {
    const size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const uint64_t a = offsets[s], b = offsets[s + 1];
    if (b < a || b > n_total || b - a >= ((uint64_t)1 << 30)) {
        set_device_error(ws_hdr, RS_ERR_INVALID_ARG, (uint32_t)s);
        return;
    }
    if (b == a) return;
    SegDesc d{};
    d.start = a;
    d.key_lo = 0;
    d.n = (uint32_t)(b - a);
    d.bits = (uint32_t)bits;
    if (tiny && d.n <= kTinyCap)
        tiny[atomicAdd(&hdr->num_tiny, 1u)] = d;
    else if (d.n <= small_cap)
        small[atomicAdd(&hdr->num_small, 1u)] = d;
    else
        append_large(large, &hdr->num_large, &hdr->total_tiles, &hdr->total_chunks, d, tile_keys);
}

// tile -> segment and chunk -> segment maps; one block per large segment.
static __global__ void k_plan_maps(const SegDesc* __restrict__ large, const SegPlanHdr* __restrict__ hdr,
                            uint32_t tile_keys, uint32_t* tile_seg, uint32_t* chunk_seg) {
    for (uint32_t li = blockIdx.x; li < hdr->num_large; li += gridDim.x) {
        const SegDesc d = large[li];
        const uint32_t nt = ceil_div_u32(d.n, tile_keys), nc = ceil_div_u32(d.n, kSegChunk);
        for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) tile_seg[d.tile0 + i] = li;
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) chunk_seg[d.chunk0 + i] = li;
    }
}

// Per-segment digit counts of `passes` digits: seg_counts[li][q][d].  One
// block per counting chunk of a large segment.  Also zeroes zero_words words
// at zero_ptr (the first pass's look-back status).  With range_hdr, a key
// whose (key - key_lo) has bits at or above the segment's `bits` is reported
// there as RS_ERR_KEY_RANGE.
template <typename KeyT, typename Digits>
__global__ void __launch_bounds__(512) k_seg_counts(const KeyT* __restrict__ keys, const SegDesc* __restrict__ large,
                                                    const SegPlanHdr* __restrict__ hdr,
                                                    const uint32_t* __restrict__ chunk_seg, Digits dg, int passes,
                                                    uint32_t bins, uint32_t* seg_counts, uint32_t* zero_ptr,
                                                    size_t zero_words, WsHeader* range_hdr) {
    extern __shared__ uint32_t s_cnt[];  // [passes][bins]
    const int tid = threadIdx.x;
    const size_t used_words = (size_t)hdr->total_tiles * bins;  // only the rows of tiles that exist
    if (zero_words > used_words) zero_words = used_words;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + tid; i < zero_words; i += (size_t)gridDim.x * blockDim.x)
        zero_ptr[i] = 0u;
    dg.init();
    const int ncnt = passes * (int)bins;
    for (uint32_t c = blockIdx.x; c < hdr->total_chunks; c += gridDim.x) {
        const uint32_t li = chunk_seg[c];
        const SegDesc d = large[li];
        const uint32_t lo = (c - d.chunk0) * kSegChunk;
        const uint32_t hi = min(d.n, lo + kSegChunk);
        __syncthreads();
        for (int i = tid; i < ncnt; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const KeyT* kp = keys + d.start;
        const KeyT klo = (KeyT)d.key_lo;
        const bool check = range_hdr && d.bits < 8 * sizeof(KeyT);
        dg.for_segment(d);
        bool bad = false;
        // eight keys per thread per step are loaded before any is counted, so
        // that enough loads are in flight to cover the memory latency
        constexpr uint32_t kU = 8;
        uint32_t i = lo + tid;
        // 8-bit digits from bit 0, one per key byte (every segmented radix
        // sort over whole bytes): digit q is byte q of the key, read with
        // compile-time shifts
        const bool bytes = Digits::kBytesCapable && dg.byte_digits() && passes <= (int)sizeof(KeyT);
        if (bytes) {
            for (; i + (kU - 1) * blockDim.x < hi; i += kU * blockDim.x) {
                KeyT x[kU];
#pragma unroll
                for (uint32_t u = 0; u < kU; ++u) x[u] = (KeyT)(__ldcs(kp + i + u * blockDim.x) - klo);
#pragma unroll
                for (uint32_t u = 0; u < kU; ++u) {
                    bad |= check && (x[u] >> (check ? d.bits : 0)) != 0;
#pragma unroll
                    for (int q = 0; q < (int)sizeof(KeyT); ++q)
                        if (q < passes) atomicAdd(&s_cnt[q * 256 + (uint32_t)((x[u] >> (8 * q)) & 0xffu)], 1u);
                }
            }
        }
        for (; i + (kU - 1) * blockDim.x < hi; i += kU * blockDim.x) {
            KeyT x[kU];
#pragma unroll
            for (uint32_t u = 0; u < kU; ++u) x[u] = (KeyT)(__ldcs(kp + i + u * blockDim.x) - klo);
#pragma unroll
            for (uint32_t u = 0; u < kU; ++u) {
                bad |= check && (x[u] >> (check ? d.bits : 0)) != 0;
                bad |= !dg.in_range(x[u]);
                if constexpr (Digits::kOneDigit)
                    atomicAdd(&s_cnt[dg(x[u], 0)], 1u);
                else
                    for (int q = 0; q < passes; ++q) atomicAdd(&s_cnt[q * bins + dg(x[u], q)], 1u);
            }
        }
        for (; i < hi; i += blockDim.x) {
            const KeyT x = (KeyT)(__ldcs(kp + i) - klo);
            bad |= check && (x >> (check ? d.bits : 0)) != 0;
            bad |= !dg.in_range(x);
            if constexpr (Digits::kOneDigit)
                atomicAdd(&s_cnt[dg(x, 0)], 1u);
            else
                for (int q = 0; q < passes; ++q) atomicAdd(&s_cnt[q * bins + dg(x, q)], 1u);
        }
        if (bad && range_hdr) set_device_error(range_hdr, RS_ERR_KEY_RANGE, li);
        __syncthreads();
        uint32_t* out = seg_counts + (size_t)li * ncnt;
        for (int i = tid; i < ncnt; i += blockDim.x)
            if (s_cnt[i]) atomicAdd(&out[i], s_cnt[i]);
    }
}

// Exclusive prefix of every (segment, pass) row of bins counts, in place.
// One block of 256 threads per row.
static __global__ void __launch_bounds__(256) k_seg_scan(uint32_t* rows, const SegPlanHdr* __restrict__ hdr, int passes,
                                                  uint32_t bins, int use_next) {
    extern __shared__ uint32_t s_row[];  // [bins] + scan scratch
    const uint32_t nrows = (use_next ? hdr->num_next : hdr->num_large) * (uint32_t)passes;
    for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
        uint32_t* row = rows + (size_t)r * bins;
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < bins; d += 256) s_row[d] = row[d];
        __syncthreads();
        block_exclusive_scan_smem<256>(s_row, (int)bins, s_row + bins);
        for (uint32_t d = threadIdx.x; d < bins; d += 256) row[d] = s_row[d];
    }
}

// Parameters of a segmented scatter pass.
template <typename DigitOp>
struct SegPassParams {
    PassParams<DigitOp> base;      // keys, values, op, status, counters, hooks (n, num_tiles unused)
    const SegDesc* segs;           // large segments
    const SegPlanHdr* hdr;         // total_tiles
    const uint32_t* tile_seg;      // global tile -> segment
    const uint32_t* seg_base;      // [segment][passes][bins] exclusive prefixes
    int pass;
    int passes;
};

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB, typename DigitOp>
__global__ void __launch_bounds__(BLOCK, MINB) k_onesweep_seg(SegPassParams<DigitOp> sp) {
    constexpr int kTile = BLOCK * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tile;
    const PassParams<DigitOp>& p = sp.base;
    const uint32_t bins = 1u << p.digit_bits;
    const PassSmem<KeyT> sm = carve_pass_smem<KeyT, VALS, BLOCK>(smem, bins, kTile);
    DigitOp op = p.op;
    op.init();
    const int tid = threadIdx.x;
    while (true) {
        for (uint32_t i = tid; i < (uint32_t)(BLOCK / 16) * sm.tab_stride; i += BLOCK) sm.tab[i] = 0u;
        if (tid == 0) s_tile = atomicAdd(p.tile_ctr, 1u);
        __syncthreads();
        const uint32_t g = s_tile;
        if (g >= sp.hdr->total_tiles) return;  // uniform across the block
        if (p.status_next)
            for (uint32_t d = tid; d < bins; d += BLOCK) p.status_next[(size_t)g * bins + d] = 0u;
        const uint32_t li = sp.tile_seg[g];
        const SegDesc seg = sp.segs[li];
        op.for_segment(seg);  // digit parameters of this segment, if they differ per segment
        const uint32_t base = (g - seg.tile0) * (uint32_t)kTile;
        TileCtx<KeyT> c;
        c.kin = static_cast<const KeyT*>(p.keys_in) + seg.start + base;
        c.vin = VALS ? p.vals_in + seg.start + base : nullptr;
        c.kout = static_cast<KeyT*>(p.keys_out) + seg.start;
        c.vout = VALS ? p.vals_out + seg.start : nullptr;
        c.digit_base = sp.seg_base + ((size_t)li * sp.passes + sp.pass) * bins;
        c.tile = g;
        c.first_tile = seg.tile0;
        c.tile_n = min((uint32_t)kTile, seg.n - base);
        c.seg_n = seg.n;
        c.key_lo = (KeyT)seg.key_lo;
        const bool publish = (int)g != p.stall_tile;
        if (c.tile_n == (uint32_t)kTile)
            onesweep_tile<KeyT, VALS, BLOCK, ITEMS, true>(p, op, sm, c, bins, publish);
        else
            onesweep_tile<KeyT, VALS, BLOCK, ITEMS, false>(p, op, sm, c, bins, publish);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Shared-memory sort of one small segment per block: load it, run stable LSD
// passes of up to 9 bits over (key - key_lo) between two shared buffers
// (each pass ranks keys inside their warps exactly like the scatter pass),
// write it back.  In bucket mode the first pass sorts by the key's bucket
// relative to the segment's first bucket (the insert step of Algorithm 2)
// and each bucket is then sorted by a stable rank sort (every key counts the
// bucket's keys that precede it: the comparisons of insertion sort,
// Algorithm 1, made for all keys at once); a segment with a bucket above
// kBucketSortMax keys, or spanning more than 256 buckets, is sorted by its
// key bits instead, which gives the same order because bucket ids grow with
// the key.  So is every segment of 32-bit keys, and a segment of 64-bit
// keys that span at most kLeafKeyBits bits: the whole run of buckets is then
// sorted by its key bits in passes of at most 9 bits, which on GB300 costs
// less than the counting pass by bucket and the rank sort of every bucket
// for runs of 32-bit keys (about 18 bits at 100M uniform keys and n/16
// buckets); for 64-bit keys, whose runs span about 49 bits, the bucket way
// wins.  The result is the same: sorting a run of whole buckets by key
// sorts every bucket and keeps them in bucket order.  For 32-bit keys the
// bucket path is compiled out, which also frees the registers it would
// hold.
constexpr uint32_t kBucketSortMax = 48;
constexpr uint32_t kLeafKeyBits = 24;

// Asynchronous copy of one 4- or 8-byte word from global to shared memory
// (no register holds it, so a thread can have all its copies in flight);
// cp_async_wait_all waits for all of the thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_word(void* smem, const void* gmem) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async of 4 or 8 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(smem)), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Rank tables of the shared-memory sort: one per half-warp, room for 9-bit
// digits (kLocalMaxBins + kSubPad 32-bit words each, as in the scatter pass).
constexpr uint32_t kLocalMaxBins = 512;
constexpr uint32_t kLocalTabStride = kLocalMaxBins + kSubPad;

template <typename KeyT, bool VALS, int BLOCK>
struct LocalSmem {
    static constexpr int kWarps = BLOCK / 32;
    static size_t bytes(int cap) {
        size_t b = (size_t)(BLOCK / 16) * (kLocalMaxBins + kSubPad) * 4;  // rank tables (one per half-warp)
        b += 2 * (size_t)cap * sizeof(KeyT);          // key buffers
        if (VALS) b += 2 * (size_t)cap * 4;           // value buffers
        b += kLocalMaxBins * 4 * 2 + (kWarps + 1 + 3) * 4 + 16;  // starts, counts, scan scratch, flags
        b += (size_t)cap;                             // bucket of each staged key (bucket mode)
        return b;
    }
};


// One stable pass of the shared-memory sort: keys (and values) move from
// (ka, va) to (kb, vb) ordered by digit dfun(key) < bins (at most 512).
// Each half-warp in use owns a contiguous run of 16 * ITEMS keys and ranks
// them with subwarp_rank; only the warps whose runs reach into the segment
// take part (a short segment leaves the other warps idle rather than
// spreading a few keys over every thread, whose empty items would still
// issue their instructions), and table work covers only the tables and
// the `bins` words in use.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, typename DFun>
__device__ __forceinline__ void local_pass(const KeyT* ka, const uint32_t* va, KeyT* kb, uint32_t* vb, uint32_t m,
                                           int dbits, uint32_t* s_tab, uint32_t* s_start, uint32_t* s_cnt,
                                           uint32_t* s_scan, DFun dfun, uint8_t* s_dig = nullptr) {
    constexpr uint32_t kRun = 16u * ITEMS;  // keys per half-warp
    const uint32_t bins = 1u << dbits;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const uint32_t nsub = 2u * ((m + 2u * kRun - 1u) / (2u * kRun));  // half-warps in use, whole warps
    for (uint32_t i = tid; i < nsub * bins; i += BLOCK)
        s_tab[(i >> dbits) * kLocalTabStride + (i & (bins - 1u))] = 0u;
    __syncthreads();
    const uint32_t sub = 2u * (uint32_t)warp + (uint32_t)half;
    const bool active = 2u * (uint32_t)warp < nsub;  // the same for the whole warp
    const uint32_t tab = smem_addr(s_tab + (size_t)sub * kLocalTabStride);
    const uint32_t hbit = 1u << hl, hlt = hbit - 1u, hgt = 0xffffu & ~(hlt | hbit);
    const uint32_t hofs = sub * kRun + (uint32_t)hl;
    // 32-bit keys stay in registers from ranking to scattering; 64-bit keys
    // are read again (holding them would spill)
    constexpr bool kKeep = sizeof(KeyT) == 4;
    uint32_t dr[ITEMS];
    KeyT kr[kKeep ? ITEMS : 1];
    if (active) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t idx = hofs + (uint32_t)i * 16u;
            const bool ok = idx < m;
            const KeyT k = ok ? ka[idx] : (KeyT)0;
            if (kKeep) kr[kKeep ? i : 0] = k;
            const uint32_t d = ok ? dfun(k) : 0u;
            dr[i] = (d << 16) | subwarp_rank<false>(tab, d, ok, hbit, hlt, hgt);
        }
    }
    __syncthreads();
    for (uint32_t d = tid; d < bins; d += BLOCK) {
        uint32_t sum = 0;
#pragma unroll 4
        for (uint32_t s = 0; s < nsub; ++s) sum += s_tab[(size_t)s * kLocalTabStride + d] >> 16;
        s_cnt[d] = sum;
        s_start[d] = sum;
    }
    __syncthreads();
    block_exclusive_scan_smem<BLOCK>(s_start, (int)bins, s_scan);
    for (uint32_t d = tid; d < bins; d += BLOCK) {
        uint32_t run = s_start[d];
#pragma unroll 4
        for (uint32_t s = 0; s < nsub; ++s) {
            uint32_t* e = s_tab + (size_t)s * kLocalTabStride + d;
            const uint32_t cnt = *e >> 16;
            *e = run;
            run += cnt;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t idx = hofs + (uint32_t)i * 16u;
            if (idx < m) {
                const uint32_t pos = ld_shared_u32(tab + 4u * (dr[i] >> 16)) + (dr[i] & 0xffffu);
                if (pos < m) {
                    kb[pos] = kKeep ? kr[kKeep ? i : 0] : ka[idx];
                    if (VALS) vb[pos] = va[idx];
                    if (s_dig) s_dig[pos] = (uint8_t)(dr[i] >> 16);
                }
            }
        }
    }
    __syncthreads();
}

// Items per lane of the shared-memory sort's passes over segments of at
// most BLOCK * RS_LOCAL_FIT_ITEMS keys (longer segments take ITEMS): a
// short segment is then spread over more warps, whose rank chains run side
// by side instead of one after another.  One such variant besides ITEMS
// keeps every instantiation free of spills.
#ifndef RS_LOCAL_FIT_ITEMS
#define RS_LOCAL_FIT_ITEMS 4
#endif

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, typename DFun>
__device__ __forceinline__ void local_pass_fit(const KeyT* ka, const uint32_t* va, KeyT* kb, uint32_t* vb, uint32_t m,
                                               int dbits, uint32_t* s_tab, uint32_t* s_start, uint32_t* s_cnt,
                                               uint32_t* s_scan, DFun dfun, uint8_t* s_dig = nullptr) {
    if (ITEMS > RS_LOCAL_FIT_ITEMS && m <= (uint32_t)BLOCK * RS_LOCAL_FIT_ITEMS)
        local_pass<KeyT, VALS, BLOCK, RS_LOCAL_FIT_ITEMS>(ka, va, kb, vb, m, dbits, s_tab, s_start, s_cnt, s_scan, dfun, s_dig);
    else
        local_pass<KeyT, VALS, BLOCK, ITEMS>(ka, va, kb, vb, m, dbits, s_tab, s_start, s_cnt, s_scan, dfun, s_dig);
}

struct LocalParams {
    const void* keys_in;
    void* keys_out;
    const uint32_t* vals_in;
    uint32_t* vals_out;
    const SegDesc* segs;
    const uint32_t* count;  // number of segments in segs; null: sort the single segment `one`
    const void* bucket;     // BucketParams (bucket mode) or null
    SegDesc one;            // the segment when count is null
    WsHeader* hdr;          // non-null: keys >= 2^bits (relative to key_lo) are reported here
    KeyXform xf;            // typed keys: sorted by their ordered image (plain sorts only)
};

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, typename BucketFn>
__global__ void __launch_bounds__(BLOCK, 3) k_local_sort(LocalParams lp, BucketFn bfn) {
    constexpr int kCap = BLOCK * ITEMS;
    constexpr int kWarps = BLOCK / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
    KeyT* kbuf[2];
    kbuf[0] = reinterpret_cast<KeyT*>(s_tab + (size_t)(BLOCK / 16) * kLocalTabStride);
    kbuf[1] = kbuf[0] + kCap;
    uint32_t* vbuf[2];
    vbuf[0] = reinterpret_cast<uint32_t*>(kbuf[1] + kCap);
    vbuf[1] = vbuf[0] + (VALS ? kCap : 0);
    uint32_t* s_start = vbuf[1] + (VALS ? kCap : 0);
    uint32_t* s_cnt = s_start + kLocalMaxBins;
    uint32_t* s_scan = s_cnt + kLocalMaxBins;
    uint32_t* s_flag = s_scan + kWarps + 1;
    uint8_t* s_dig = reinterpret_cast<uint8_t*>(s_flag + 4);

    if (bfn.active()) bfn.init();
    const uint32_t nseg = lp.count ? *lp.count : 1u;
    for (uint32_t si = blockIdx.x; si < nseg; si += gridDim.x) {
        const SegDesc seg = lp.count ? lp.segs[si] : lp.one;
        const uint32_t m = seg.n;
        const KeyT klo = (KeyT)seg.key_lo;
        bfn.for_segment(seg);
        __syncthreads();
        const KeyT* kin = static_cast<const KeyT*>(lp.keys_in) + seg.start;
        // the segment this block takes next is asked into L2 now, so that
        // its copies below wait on L2 rather than on DRAM (items of 8 bytes
        // or more: 4096-key segments with values 1.285 -> 1.237 ms per 100M
        // keys; no gain for 4-byte keys alone)
        if (sizeof(KeyT) + (VALS ? 4 : 0) >= 8 && lp.count && si + gridDim.x < nseg) {
            const SegDesc nx = lp.segs[si + gridDim.x];
            const char* kb = reinterpret_cast<const char*>(static_cast<const KeyT*>(lp.keys_in) + nx.start);
            for (uint32_t i = threadIdx.x; i < (nx.n * (uint32_t)sizeof(KeyT) + 127u) / 128u; i += BLOCK)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(kb + (size_t)i * 128));
            if (VALS) {
                const char* vb = reinterpret_cast<const char*>(lp.vals_in + nx.start);
                for (uint32_t i = threadIdx.x; i < (nx.n * 4u + 127u) / 128u; i += BLOCK)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(vb + (size_t)i * 128));
            }
        }
        bool bad = false;
        const bool xf = lp.xf.active();
        // the segment comes in by asynchronous copies, all of a thread's in
        // flight at once (one memory latency per segment, no registers)
        for (uint32_t i = threadIdx.x; i < m; i += BLOCK) {
            cp_async_word<sizeof(KeyT)>(&kbuf[0][i], kin + i);
            if (VALS) cp_async_word<4>(&vbuf[0][i], lp.vals_in + seg.start + i);
        }
        cp_async_wait_all();
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += BLOCK) {
            KeyT k = kbuf[0][i];
            if (xf) {
                k = lp.xf.to_ordered(k);
                kbuf[0][i] = k;
            }
            bad |= seg.bits < 8 * sizeof(KeyT) && ((KeyT)(k - klo) >> seg.bits) != 0;
            bad |= !bfn.in_range(k);
        }
        if (bad && lp.hdr) set_device_error(lp.hdr, RS_ERR_KEY_RANGE, si);
        // keys already in nondecreasing order (a sorted run) are their own
        // stable sort: nothing to rank or move.  On unsorted keys nearly every
        // thread stops at its first pair.
        if (xf) __syncthreads();
        bool in_order = true;
        for (uint32_t i = threadIdx.x; i + 1 < m && in_order; i += BLOCK) in_order = !(kbuf[0][i + 1] < kbuf[0][i]);
        const bool already_sorted = __syncthreads_and(in_order) != 0;
        int cur = 0;
        bool by_keys = !already_sorted;
        if (already_sorted) {
            // output straight from the loaded keys
        } else if (sizeof(KeyT) > 4 && bfn.active() && seg.bits > kLeafKeyBits) {
            const uint64_t b_lo = bfn.first_bucket(seg), span = bfn.bucket_span(seg);
            if (threadIdx.x == 0) *s_flag = 0u;
            __syncthreads();
            if (span <= 256) {
                local_pass_fit<KeyT, VALS, BLOCK, ITEMS>(
                    kbuf[0], vbuf[0], kbuf[1], vbuf[1], m, 8, s_tab, s_start, s_cnt, s_scan,
                    [&](KeyT k) { return (uint32_t)(bfn.bucket(k) - b_lo); }, s_dig);
                cur = 1;
                for (uint32_t d = threadIdx.x; d < 256; d += BLOCK)
                    if (s_cnt[d] > kBucketSortMax) *s_flag = 1u;
                __syncthreads();
                if (*s_flag == 0u) {
                    by_keys = false;
                    // sort every bucket: each key's place in its bucket is the
                    // number of the bucket's keys that precede it in the
                    // stable order (smaller, or equal and earlier in input
                    // order, which the counting pass kept) -- the comparisons
                    // of insertion sort (Algorithm 1), made for all keys at
                    // once instead of one bucket per thread
                    // When the run's key bits leave room for 12 more, each key
                    // is first rewritten in place as ((key - lo) << 12) | its
                    // position, which orders keys the stable way in one
                    // comparison: then a key's rank is the number of its
                    // bucket's words below its own (ties cannot occur), and
                    // the key comes back as (word >> 12) + lo.
                    const bool packed = seg.bits + 12u <= 8u * sizeof(KeyT);
                    if (packed) {
                        for (uint32_t j = threadIdx.x; j < m; j += BLOCK)
                            kbuf[1][j] = (KeyT)(((KeyT)(kbuf[1][j] - klo) << 12) | (KeyT)j);
                        __syncthreads();
                    }
                    for (uint32_t j = threadIdx.x; j < m; j += BLOCK) {
                        const KeyT key = kbuf[1][j];
                        const uint32_t d = s_dig[j];
                        const uint32_t lo = s_start[d], hi = lo + s_cnt[d];
                        uint32_t r = 0, q = lo;
                        if (packed) {
                            for (; q + 4 <= hi; q += 4)  // four independent reads per step
                                r += (kbuf[1][q] < key) + (kbuf[1][q + 1] < key) + (kbuf[1][q + 2] < key) +
                                     (kbuf[1][q + 3] < key);
                            for (; q < hi; ++q) r += kbuf[1][q] < key;
                        } else {
                            for (; q + 4 <= hi; q += 4) {
                                const KeyT o0 = kbuf[1][q], o1 = kbuf[1][q + 1], o2 = kbuf[1][q + 2],
                                           o3 = kbuf[1][q + 3];
                                r += ((o0 < key) | ((o0 == key) & (q < j))) +
                                     ((o1 < key) | ((o1 == key) & (q + 1 < j))) +
                                     ((o2 < key) | ((o2 == key) & (q + 2 < j))) +
                                     ((o3 < key) | ((o3 == key) & (q + 3 < j)));
                            }
                            for (; q < hi; ++q) {
                                const KeyT other = kbuf[1][q];
                                r += (other < key) | ((other == key) & (q < j));
                            }
                        }
                        kbuf[0][lo + r] = packed ? (KeyT)((key >> 12) + klo) : key;
                        if (VALS) vbuf[0][lo + r] = vbuf[1][j];
                    }
                    cur = 0;
                    __syncthreads();
                }
            } else {
                __syncthreads();
            }
        } else {
            __syncthreads();
        }
        if (by_keys) {
            // the fewest passes of at most 9 bits that cover the segment's
            // key bits, the bits shared evenly (18 bits: two 9-bit passes
            // instead of three 8-bit ones); the last pass takes only the
            // bits left (17 bits: 9 + 8), so its tables are no wider than
            // its digits
            const uint32_t nb = seg.bits;
            const uint32_t P = nb ? (nb + 8) / 9 : 0;
            const int dw = P ? (int)((nb + P - 1) / P) : 0;
            for (uint32_t q = 0, shift = 0; q < P; ++q, shift += (uint32_t)dw) {
                const int w = q + 1 == P ? (int)(nb - shift) : dw;
                const uint32_t dmask = (1u << w) - 1u;
                local_pass_fit<KeyT, VALS, BLOCK, ITEMS>(
                    kbuf[cur], vbuf[cur], kbuf[cur ^ 1], vbuf[cur ^ 1], m, w, s_tab, s_start, s_cnt, s_scan,
                    [&](KeyT k) { return (uint32_t)((KeyT)(k - klo) >> shift) & dmask; });
                cur ^= 1;
            }
        }
        KeyT* kout = static_cast<KeyT*>(lp.keys_out) + seg.start;
        for (uint32_t i = threadIdx.x; i < m; i += BLOCK) {
            kout[i] = xf ? lp.xf.from_ordered(kbuf[cur][i]) : kbuf[cur][i];
            if (VALS) lp.vals_out[seg.start + i] = vbuf[cur][i];
        }
        __syncthreads();
    }
}

// One tiny segment ranked by one warp with KPL keys per lane (KPL * 32 >= m):
// each lane's keys are compared with every key of the segment in the warp's
// shared-memory row (the same word for every lane: a broadcast), four at a
// time; a key's rank is the number of keys before it in stable order
// (smaller, or equal and earlier), and the key (and its value) is written
// there.
template <int KPL, typename KeyT, bool VALS>
__device__ __forceinline__ void rank_tiny(const KeyT* row, uint32_t m, const KeyT (&k)[kTinyCap / 32],
                                          const uint32_t (&v)[VALS ? kTinyCap / 32 : 1], KeyT* kout,
                                          uint32_t* vout, int lane) {
    uint32_t r[KPL];
#pragma unroll
    for (int j = 0; j < KPL; ++j) r[j] = 0;
    uint32_t q = 0;
    for (; q + 4 <= m; q += 4) {
        const KeyT o0 = row[q], o1 = row[q + 1], o2 = row[q + 2], o3 = row[q + 3];
#pragma unroll
        for (int j = 0; j < KPL; ++j) {
            const uint32_t i = (uint32_t)j * 32 + lane;
            r[j] += ((o0 < k[j]) | ((o0 == k[j]) & (q < i))) + ((o1 < k[j]) | ((o1 == k[j]) & (q + 1 < i))) +
                    ((o2 < k[j]) | ((o2 == k[j]) & (q + 2 < i))) + ((o3 < k[j]) | ((o3 == k[j]) & (q + 3 < i)));
        }
    }
    for (; q < m; ++q) {
        const KeyT o = row[q];
#pragma unroll
        for (int j = 0; j < KPL; ++j) r[j] += (o < k[j]) | ((o == k[j]) & (q < (uint32_t)j * 32 + lane));
    }
#pragma unroll
    for (int j = 0; j < KPL; ++j) {
        const uint32_t i = (uint32_t)j * 32 + lane;
        if (i < m && r[j] < m) {
            kout[r[j]] = k[j];
            if (VALS) vout[r[j]] = v[j];
        }
    }
}

// One tiny segment sorted by one warp with a bitonic network (Batcher 1968)
// over N = 32 * KPL slots, KPL per lane: slot lane * KPL + r holds the key
// loaded as item r (input position r * 32 + lane).  Slots past the segment
// hold the largest key.  Pairs KPL or more slots apart are exchanged between
// lanes, nearer pairs inside a lane.  Keys compare by (key, input position),
// a total order, so the sort is stable: equal keys keep their input order,
// and each value is fetched from its key's input position at the end (all
// reads before the first write, so the sort may run in place).  For
// keys only the position is not needed (equal keys are indistinguishable).
// Costs O(m log^2 m) comparisons against rank_tiny's O(m^2).
template <int KPL, typename KeyT, bool VALS>
__device__ __forceinline__ void bitonic_tiny(uint32_t m, const KeyT (&k)[kTinyCap / 32], const uint32_t* vin,
                                             KeyT* kout, uint32_t* vout, int lane) {
    constexpr int N = 32 * KPL;
    KeyT a[KPL];
    uint32_t ix[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t i = (uint32_t)r * 32 + lane;
        a[r] = i < m ? k[r] : ~(KeyT)0;
        ix[r] = i;
    }
    // x before y in (key, position) order (keys only: by key)
    auto before = [](KeyT x, uint32_t xi, KeyT y, uint32_t yi) {
        return VALS ? (x < y || (x == y && xi < yi)) : x < y;
    };
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j < KPL) {
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    if ((r & j) == 0) {
                        const int r2 = r | j;
                        const bool up = (((uint32_t)lane * KPL + r) & kk) == 0;
                        const bool sw = up ? before(a[r2], ix[r2], a[r], ix[r]) : before(a[r], ix[r], a[r2], ix[r2]);
                        if (sw) {
                            const KeyT t = a[r];
                            a[r] = a[r2];
                            a[r2] = t;
                            const uint32_t ti = ix[r];
                            ix[r] = ix[r2];
                            ix[r2] = ti;
                        }
                    }
                }
            } else {
                const int lj = j / KPL;
#pragma unroll
                for (int r = 0; r < KPL; ++r) {
                    const KeyT o = __shfl_xor_sync(0xffffffffu, a[r], lj);
                    const uint32_t oi = VALS ? __shfl_xor_sync(0xffffffffu, ix[r], lj) : 0u;
                    const uint32_t e = (uint32_t)lane * KPL + r;
                    const bool lower = (e & j) == 0, up = (e & kk) == 0;
                    // the lower slot of an ascending pair keeps the earlier key
                    const bool take = lower == up ? before(o, oi, a[r], ix[r]) : before(a[r], ix[r], o, oi);
                    if (take) {
                        a[r] = o;
                        ix[r] = oi;
                    }
                }
            }
        }
    }
    // every value is read before any is written: in place, vout is vin
    uint32_t vv[VALS ? KPL : 1];
    if (VALS) {
#pragma unroll
        for (int r = 0; r < KPL; ++r) vv[r] = ((uint32_t)lane * KPL + r) < m ? vin[ix[r]] : 0u;
        __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
        const uint32_t e = (uint32_t)lane * KPL + r;
        if (e < m) {
            kout[e] = a[r];
            if (VALS) vout[e] = vv[r];
        }
    }
}

// Warp sort of tiny segments: each warp takes segments of at most kTinyCap
// keys from the list.  Segments of at most 32 keys are ranked against the
// warp's shared-memory row (rank_tiny), larger ones go through a bitonic
// network in registers (bitonic_tiny).  Keys at or above 2^bits are reported
// in hdr.
template <typename KeyT, bool VALS>
__global__ void __launch_bounds__(256, VALS ? 2 : 4) k_tiny_sort(const KeyT* __restrict__ keys_in, KeyT* keys_out,
                                                   const uint32_t* __restrict__ vals_in, uint32_t* vals_out,
                                                   const SegDesc* __restrict__ segs, const uint32_t* count,
                                                   WsHeader* hdr) {
    constexpr int kWarps = 256 / 32, kPerLane = kTinyCap / 32;
    __shared__ KeyT s_keys[kWarps][kTinyCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    KeyT* row = s_keys[warp];
    const uint32_t nseg = *count;
    const uint32_t stride = gridDim.x * kWarps;
    bool bad = false;
    // software pipeline: the next segment's descriptor and keys are loaded
    // before the current one is sorted, so their latency overlaps the sort
    SegDesc nsd{};
    KeyT nk[kPerLane];
    auto load = [&](uint32_t at) {
        nsd = segs[at];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            const uint32_t i = (uint32_t)j * 32 + lane;
            nk[j] = i < nsd.n ? keys_in[nsd.start + i] : (KeyT)0;
        }
    };
    uint32_t si = blockIdx.x * kWarps + warp;
    if (si < nseg) load(si);
    for (; si < nseg; si += stride) {
        const SegDesc sd = nsd;
        const uint32_t m = sd.n;
        KeyT k[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            k[j] = nk[j];
            if ((uint32_t)j * 32 + lane < m) bad |= sd.bits < 8 * sizeof(KeyT) && (k[j] >> sd.bits) != 0;
        }
        if (si + stride < nseg) load(si + stride);
        KeyT* kout = keys_out + sd.start;
        uint32_t* vout = VALS ? vals_out + sd.start : nullptr;
        const uint32_t* vin = VALS ? vals_in + sd.start : nullptr;
        if (m <= 32) {
            // rank_tiny with one key per lane reads the keys from the row
            uint32_t v[VALS ? kPerLane : 1] = {};
            if (lane < (int)m) {
                row[lane] = k[0];
                if (VALS) v[0] = vin[lane];
            }
            __syncwarp();
            rank_tiny<1, KeyT, VALS>(row, m, k, v, kout, vout, lane);
        } else if (m <= 64) {
            bitonic_tiny<2, KeyT, VALS>(m, k, vin, kout, vout, lane);
        } else if (m <= 128) {
            bitonic_tiny<4, KeyT, VALS>(m, k, vin, kout, vout, lane);
        } else {
            bitonic_tiny<8, KeyT, VALS>(m, k, vin, kout, vout, lane);
        }
        __syncwarp();
    }
    if (bad && hdr) set_device_error(hdr, RS_ERR_KEY_RANGE, blockIdx.x);
}

// Bucket function placeholder for plain segmented sorts (no bucket step).
struct NoBucket {
    __device__ __forceinline__ bool active() const { return false; }
    __device__ __forceinline__ void init() {}
    __device__ __forceinline__ void for_segment(const SegDesc&) {}
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT) const {
        return true;
    }
    __device__ __forceinline__ uint64_t first_bucket(const SegDesc&) const { return 0; }
    __device__ __forceinline__ uint64_t bucket_span(const SegDesc&) const { return 0; }
    template <typename KeyT>
    __device__ __forceinline__ uint64_t bucket(KeyT) const {
        return 0;
    }
};

}  // namespace rs
