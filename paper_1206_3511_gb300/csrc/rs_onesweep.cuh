// rs_onesweep.cuh -- the two kernels of one LSD radix sort on the GPU.
//
//  k_digit_counts: the counting loop of the counting sort (Sec. 2.4,
//    Algorithm 3) for every pass of the radix sort (Sec. 2.5, Algorithm 4) in
//    one read of the keys; the last block turns the counts into exclusive
//    prefixes, which are the counting sort's "number of smaller digits".
//    For radix sorts it also checks whether the keys are already in order,
//    and if so writes prefixes that send every pass down its copy path.
//
//  k_onesweep: one stable counting-sort pass (the placement loop of Algorithm
//    3) done block-wise, in the manner of Onesweep (Adinets & Merrill,
//    arXiv:2206.01784): each block takes the next tile (dynamic tile id),
//    ranks its keys stably by digit inside each half-warp (lane masks built
//    with shared-memory atomic OR in a per-half-warp table of packed mask and
//    count words, see subwarp_rank), obtains the
//    number of equal digits in all earlier tiles through a decoupled
//    look-back over per-(tile, digit) status words, and writes each key to
//    digit_base[d] + (earlier tiles' d) + (rank inside the tile).  The keys
//    are read once and written once per pass.  A pass whose keys all carry
//    one digit copies its input (identity_pass); a warp whose keys all carry
//    one digit ranks them by position.
#pragma once

#include "rs_common.cuh"

namespace rs {

// Digit of a key for plain LSD radix sort: (key >> shift) & mask.
struct RadixDigit {
    static constexpr bool kStageDigit = false;  // the digit is two operations: recompute it when scattering
    int shift;
    uint32_t mask;
    __device__ __forceinline__ void init() {}
    template <typename Seg>
    __device__ __forceinline__ void for_segment(const Seg&) {}
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT k) const {
        return (uint32_t)(k >> shift) & mask;
    }
    // every key in [lo, hi] has one digit: their bits from the digit up agree
    template <typename KeyT>
    __device__ __forceinline__ bool same_digit_range(KeyT lo, KeyT hi) const {
        return (lo >> shift) == (hi >> shift);
    }
};

template <typename T>
__device__ __forceinline__ T warp_min(T x) {
    if constexpr (sizeof(T) == 4) {
        return __reduce_min_sync(0xffffffffu, x);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y < x ? y : x;
        }
        return x;
    }
}

template <typename T>
__device__ __forceinline__ T warp_max(T x) {
    if constexpr (sizeof(T) == 4) {
        return __reduce_max_sync(0xffffffffu, x);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y > x ? y : x;
        }
        return x;
    }
}

// ---------------------------------------------------------------------------
// Digit counts of every pass in one read.

// Digit q of a key for the counting kernels: (x >> (shift0 + q*D)) & mask,
// and the key-range check (every key must be below 2^key_bits).
struct RadixDigits {
    static constexpr bool kBytesCapable = true;
    static constexpr bool kOneDigit = false;
    int shift0;
    int digit_bits;
    uint32_t mask;
    int key_bits;
    __device__ __forceinline__ void init() {}
    template <typename Seg>
    __device__ __forceinline__ void for_segment(const Seg&) {}
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT x, int q) const {
        return (uint32_t)(x >> (shift0 + q * digit_bits)) & mask;
    }
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT k) const {
        return key_bits >= (int)(8 * sizeof(KeyT)) || (k >> key_bits) == 0;
    }
    // the order the sort produces: by the key itself
    template <typename KeyT>
    __device__ __forceinline__ KeyT order(KeyT k) const {
        return k;
    }
    // digit q is byte q of order(k) (8-bit digits from bit 0)
    __host__ __device__ bool byte_digits() const { return shift0 == 0 && digit_bits == 8; }
};

// RadixDigits of the ordered image of typed keys (signed, float, descending):
// every key is mapped by to_ordered before its digits are taken; all 2^w
// images are valid, so there is no range check.
struct OrderedRadixDigits {
    static constexpr bool kBytesCapable = true;
    static constexpr bool kOneDigit = false;
    RadixDigits base;
    KeyXform xf;
    __device__ __forceinline__ void init() {}
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT x, int q) const {
        return base(xf.to_ordered(x), q);
    }
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT) const {
        return true;
    }
    // the order the sort produces: by the ordered image
    template <typename KeyT>
    __device__ __forceinline__ KeyT order(KeyT k) const {
        return xf.to_ordered(k);
    }
    __host__ __device__ bool byte_digits() const { return base.byte_digits(); }
};

struct CountParams {
    const void* keys;
    size_t n;
    int passes;        // P
    uint32_t bins;     // 2^D
    uint32_t* counts;  // [P][bins], zero on entry
    uint32_t* scan;    // [P][bins] exclusive prefixes (nullable)
    uint32_t* zero_ptr;  // words zeroed by the kernel (first pass's status words)
    size_t zero_words;
    WsHeader* hdr;
    uint32_t* unsorted;  // nonnull: set nonzero if some key is above the next one (in dg's order)
};

constexpr int kCountBlock = 512;
constexpr int kCountVecIters = 8;  // 16-byte loads per thread per chunk

// BYTES: digit q is byte q of dg.order(k) (8-bit digits from bit 0, the
// usual case): the key is mapped once and every digit is a fixed byte.
template <typename KeyT, typename Digits, bool BYTES>
__device__ __forceinline__ void count_key(uint32_t* s_cnt, KeyT k, const Digits& dg, int P, uint32_t bins,
                                          bool& bad) {
    bad |= !dg.in_range(k);
    if constexpr (Digits::kOneDigit) {  // one digit per key (the bucket sort's partition digit)
        atomicAdd(&s_cnt[dg(k, 0)], 1u);
    } else if (BYTES) {
        const KeyT o = dg.order(k);
#pragma unroll
        for (int q = 0; q < (int)sizeof(KeyT); ++q)
            if (q < P) atomicAdd(&s_cnt[q * 256 + (uint32_t)((o >> (8 * q)) & 0xffu)], 1u);
    } else {
        for (int q = 0; q < P; ++q) atomicAdd(&s_cnt[q * bins + dg(k, q)], 1u);
    }
}

template <typename KeyT, typename Digits, bool BYTES = false>
__global__ void __launch_bounds__(kCountBlock) k_digit_counts(CountParams p, Digits dg) {
    extern __shared__ uint32_t s_cnt[];  // [P][bins], then kCountBlock/32+1 scan words
    __shared__ uint32_t s_last;
    const uint32_t bins = p.bins;
    const int ncnt = p.passes * (int)bins;
    uint32_t* s_scan = s_cnt + ncnt;
    const int tid = threadIdx.x;
    dg.init();
    for (int i = tid; i < ncnt; i += kCountBlock) s_cnt[i] = 0;
    for (size_t i = (size_t)blockIdx.x * kCountBlock + tid; i < p.zero_words; i += (size_t)gridDim.x * kCountBlock)
        p.zero_ptr[i] = 0;
    __syncthreads();

    // keys before the first 16-byte boundary and after the last one are
    // counted one by one; the body in between with 16-byte loads
    constexpr int kPerVec = 16 / sizeof(KeyT);
    const KeyT* keys = static_cast<const KeyT*>(p.keys);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    size_t head = ((16 - (addr & 15)) & 15) / sizeof(KeyT);
    if (head > p.n) head = p.n;
    const size_t nvec = (p.n - head) / kPerVec;
    const size_t tail0 = head + nvec * kPerVec;
    bool bad = false;
    // with p.unsorted: is every key at most the next one?  Each key is
    // compared with its successor, wherever that is loaded.
    const bool check = p.unsorted != nullptr;
    bool inv = false;
    const size_t gthreads = (size_t)gridDim.x * kCountBlock;
    const size_t gtid = (size_t)blockIdx.x * kCountBlock + tid;
    // (a thread stops checking at its first inversion: on unordered keys
    // that is its first few keys)
    for (size_t i = gtid; i < head; i += gthreads) {
        count_key<KeyT, Digits, BYTES>(s_cnt, keys[i], dg, p.passes, bins, bad);
        if (check && !inv && i + 1 < p.n) inv = dg.order(keys[i + 1]) < dg.order(keys[i]);
    }
    for (size_t i = tail0 + gtid; i < p.n; i += gthreads) {
        count_key<KeyT, Digits, BYTES>(s_cnt, keys[i], dg, p.passes, bins, bad);
        if (check && !inv && i + 1 < p.n) inv = dg.order(keys[i + 1]) < dg.order(keys[i]);
    }
    const uint4* vec = reinterpret_cast<const uint4*>(keys + head);
    constexpr size_t kChunk = (size_t)kCountBlock * kCountVecIters;
    for (size_t base = (size_t)blockIdx.x * kChunk; base < nvec; base += (size_t)gridDim.x * kChunk) {
        uint4 v[kCountVecIters];
#pragma unroll
        for (int j = 0; j < kCountVecIters; ++j) {
            const size_t idx = base + (size_t)j * kCountBlock + tid;
            v[j] = idx < nvec ? __ldcs(vec + idx) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < kCountVecIters; ++j) {
            const size_t idx = base + (size_t)j * kCountBlock + tid;
            if (idx < nvec) {
                const KeyT* kk = reinterpret_cast<const KeyT*>(&v[j]);
#pragma unroll
                for (int e = 0; e < kPerVec; ++e) count_key<KeyT, Digits, BYTES>(s_cnt, kk[e], dg, p.passes, bins, bad);
                if (check && !inv) {
#pragma unroll
                    for (int e = 0; e + 1 < kPerVec; ++e) inv |= dg.order(kk[e + 1]) < dg.order(kk[e]);
                    const size_t nxt = head + (idx + 1) * kPerVec;  // the key after this vector
                    if (!inv && nxt < p.n) inv = dg.order(keys[nxt]) < dg.order(kk[kPerVec - 1]);
                }
            }
        }
    }
    if (bad) set_device_error(p.hdr, RS_ERR_KEY_RANGE, blockIdx.x);
    if (__syncthreads_or(inv) && tid == 0) atomicOr(p.unsorted, 1u);
    for (int i = tid; i < ncnt; i += kCountBlock)
        if (s_cnt[i]) atomicAdd(&p.counts[i], s_cnt[i]);

    if (!p.scan) return;
    // the last block to finish turns the counts into exclusive prefixes
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.hdr->done_ctr[0], 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // Keys already in order are their own stable sort.  Then every pass's
    // prefixes are written as if all keys carried the first key's digit, so
    // that every pass takes its copy path: the copies carry the input to the
    // output unchanged (and the typed-key mapping there and back).
    const bool in_order = p.unsorted && __ldcg(p.unsorted) == 0u;
    const KeyT k0 = static_cast<const KeyT*>(p.keys)[0];
    for (int q = 0; q < p.passes; ++q) {
        if (in_order) {
            const uint32_t d0 = dg(k0, q);
            for (uint32_t d = tid; d < bins; d += kCountBlock) p.scan[q * bins + d] = d <= d0 ? 0u : (uint32_t)p.n;
            continue;
        }
        for (uint32_t d = tid; d < bins; d += kCountBlock) s_cnt[d] = __ldcg(&p.counts[q * bins + d]);
        __syncthreads();
        block_exclusive_scan_smem<kCountBlock>(s_cnt, (int)bins, s_scan);
        for (uint32_t d = tid; d < bins; d += kCountBlock) p.scan[q * bins + d] = s_cnt[d];
        __syncthreads();
    }
}

inline size_t count_smem_bytes(int passes, int digit_bits) {
    return ((size_t)passes * ((size_t)1 << digit_bits) + kCountBlock / 32 + 1) * sizeof(uint32_t);
}

// Largest digit-count shared memory over every digit width and 64-bit keys.
inline size_t max_count_smem_bytes() {
    size_t best = 0;
    for (int D = kMinDigitBits; D <= kMaxDigitBits; ++D) {
        size_t b = count_smem_bytes((64 + D - 1) / D, D);
        if (b > best) best = b;
    }
    return best;
}

// ---------------------------------------------------------------------------
// One stable scatter pass.
template <typename DigitOp>
struct PassParams {
    const void* keys_in;
    void* keys_out;
    const uint32_t* vals_in;
    uint32_t* vals_out;
    uint32_t n;
    uint32_t num_tiles;
    int digit_bits;
    DigitOp op;
    const uint32_t* digit_base;  // [bins] exclusive prefix of this pass's digit counts
    uint32_t* status;            // [num_tiles][bins], zero on entry
    uint32_t* status_next;       // [num_tiles][bins] zeroed here for the next pass (nullable)
    uint32_t* tile_ctr;          // dynamic tile counter, zero on entry
    WsHeader* hdr;
    uint32_t spin_limit;
    int stall_tile;              // test hook: this tile never publishes (-1 = off)
    KeyXform xf;                 // typed keys: map loaded keys to their ordered image (xf_in) and
    int xf_in, xf_out;           // stored keys back (xf_out); both 0 for unsigned keys
};

// Rank tables of a scatter-pass block: one per half-warp ("sub"), each of
// bins + kSubPad 32-bit words (the pad staggers the tables across banks).
constexpr uint32_t kSubPad = 4;

template <typename KeyT, bool VALS, int BLOCK, int ITEMS>
struct OnesweepShape {
    static constexpr int kWarps = BLOCK / 32;
    static constexpr int kSubs = BLOCK / 16;
    static constexpr int kTile = BLOCK * ITEMS;
    static_assert(kTile < 65536, "tile offsets are 16-bit");
    static_assert(16 * ITEMS < 65536, "a half-warp's digit count is 16-bit");
    static size_t smem_bytes(int digit_bits) {
        const size_t bins = (size_t)1 << digit_bits;
        size_t b = (size_t)kSubs * (bins + kSubPad) * 4;  // per-half-warp rank tables
        b += (size_t)kTile * sizeof(KeyT);     // staged keys
        if (VALS) b += (size_t)kTile * 4;      // staged values
        b += bins * 4 * 2;                     // local starts, scatter deltas
        b += (kWarps + 1 + 3) * 4;             // scan scratch
        return b;
    }
};

// Stable rank of one key among the keys of its half-warp that carry the
// same digit, in the half-warp's order (items in order, lanes in order within
// an item).  Entry d of the half-warp's table (one 32-bit word at tab + 4d):
// low 16 bits = peer mask of the item being ranked, one bit per lane of the
// half-warp (built with shared atomic OR, so the mask does not depend on the
// order in which the hardware applies the ORs), high 16 bits = number of keys
// with digit d in the half-warp's earlier items.  The highest lane of each
// peer group advances the count and clears the mask with one store.  One
// word per entry spreads the 32 lanes' accesses over all 32 banks, and the
// count comes with the mask in the same load.
template <bool ALL>
__device__ __forceinline__ uint32_t subwarp_rank(uint32_t tab, uint32_t d, bool ok, uint32_t hbit, uint32_t hlt,
                                                 uint32_t hgt) {
    const uint32_t addr = tab + 4u * d;
    if (ALL)
        asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(addr), "r"(hbit) : "memory");
    else
        red_or_shared_if(addr, hbit, ok);
    __syncwarp();
    const uint32_t e = ld_shared_u32(addr);
    __syncwarp();
    const uint32_t peers = (ALL || ok) ? (e & 0xffffu) : 0u;
    st_shared_u32_if(addr, ((e >> 16) + __popc(peers)) << 16, (ALL || ok) && (peers & hgt) == 0);
    __syncwarp();
    return (e >> 16) + __popc(peers & hlt);
}

// Stable rank of one key among the keys of its warp that carry the same
// digit, in warp order (items in order, lanes in order within an item).
// Entry d of the warp's table (8 bytes at tab + 8d): low word = peer mask of
// the item being ranked (built with shared atomic OR, so the mask does not
// depend on the order in which the hardware applies the ORs), high word =
// number of keys with digit d in the warp's earlier items.  The highest lane
// of each peer group advances the count and clears the mask.
template <bool ALL>
__device__ __forceinline__ uint32_t warp_rank(uint32_t tab, uint32_t d, bool ok, uint32_t lanebit, uint32_t lt,
                                              uint32_t gt) {
    const uint32_t addr = tab + 8u * d;
    if (ALL)
        asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(addr), "r"(lanebit) : "memory");
    else
        red_or_shared_if(addr, lanebit, ok);
    __syncwarp();
    const uint2 e = ld_shared_v2(addr);
    __syncwarp();
    const uint32_t peers = (ALL || ok) ? e.x : 0u;
    st_shared_v2_if(addr, 0u, e.y + __popc(peers), (ALL || ok) && (peers & gt) == 0);
    __syncwarp();
    return e.y + __popc(peers & lt);
}

// Decoupled look-back for one digit: the number of keys with digit d in the
// tiles first_tile .. tile-1.  The status words of kLookbackWindow earlier
// tiles are read per round trip (independent loads); their counts are added
// from the nearest tile backwards until the first inclusive prefix.  A tile
// whose word is still invalid is waited for (bounded: after spin_limit polls
// the error is recorded and the partial sum, which never exceeds the true
// prefix, is returned).
constexpr int kLookbackWindow = 4;

__device__ __forceinline__ uint32_t lookback_digit(const uint32_t* status, uint32_t tile, uint32_t first_tile,
                                                   uint32_t bins, uint32_t d, uint32_t spin_limit, WsHeader* hdr) {
    uint32_t excl = 0;
    int64_t t = (int64_t)tile - 1;  // nearest tile not yet added
    const int64_t lo = first_tile;
    uint32_t polls = 0;
    while (t >= lo) {
        uint32_t w[kLookbackWindow];
#pragma unroll
        for (int j = 0; j < kLookbackWindow; ++j)
            w[j] = (t - j >= lo) ? ld_relaxed(status + (size_t)(t - j) * bins + d) : kFlagPrefix;
        bool done = false, blocked = false;
        int used = 0;
#pragma unroll
        for (int j = 0; j < kLookbackWindow; ++j) {
            if (!done && !blocked) {
                const uint32_t flag = w[j] & ~kCountMask;
                if (flag == kFlagInvalid) {
                    blocked = true;
                } else {
                    excl += w[j] & kCountMask;
                    ++used;
                    done = flag == kFlagPrefix;
                }
            }
        }
        if (done) break;
        t -= used;
        if (blocked) {
            if (++polls > spin_limit) {
                set_device_error(hdr, RS_ERR_DEVICE_TIMEOUT, tile);
                break;
            }
            if (polls > 8) __nanosleep(polls < 256 ? 64 : 512);
        }
    }
    return excl;
}

// Shared-memory layout of one scatter-pass block.
template <typename KeyT>
struct PassSmem {
    uint32_t* tab;            // [subs][bins + kSubPad] rank tables, later each sub's offset per digit
    uint32_t tab_stride;      // words per sub table
    KeyT* keys;               // [tile] staged keys
    uint32_t* vals;           // [tile] staged values
    uint32_t* local;          // [bins] start of each digit inside the staged tile
    uint32_t* delta;          // [bins] segment position minus staged position
    uint32_t* scan;           // [warps + 1] block-scan scratch
    uint8_t* digs;            // [tile] digit of each staged key (digit functions with kStageDigit)
};

// Shared memory of a pass: the shape's, plus one byte per key of the tile
// for digit functions that stage their digit (kStageDigit: a bucket id costs
// more than a byte stored and loaded again).
template <typename Shape, typename DigitOp>
size_t pass_smem_bytes(int digit_bits) {
    return Shape::smem_bytes(digit_bits) + (DigitOp::kStageDigit ? (size_t)Shape::kTile : 0);
}

template <typename KeyT, bool VALS, int BLOCK>
__device__ __forceinline__ PassSmem<KeyT> carve_pass_smem(unsigned char* smem, uint32_t bins, int tile_keys) {
    PassSmem<KeyT> sm;
    sm.tab = reinterpret_cast<uint32_t*>(smem);
    sm.tab_stride = bins + kSubPad;
    sm.keys = reinterpret_cast<KeyT*>(sm.tab + (size_t)(BLOCK / 16) * sm.tab_stride);
    sm.vals = reinterpret_cast<uint32_t*>(sm.keys + tile_keys);
    sm.local = sm.vals + (VALS ? tile_keys : 0);
    sm.delta = sm.local + bins;
    sm.scan = sm.delta + bins;
    sm.digs = reinterpret_cast<uint8_t*>(sm.scan + BLOCK / 32 + 4);
    return sm;
}

// What one tile works on: its keys (already offset to the tile), the output
// of its segment (positions are relative to the segment), the segment's
// digit bases, and the range of tiles its look-back may visit.
template <typename KeyT>
struct TileCtx {
    const KeyT* kin;
    const uint32_t* vin;
    KeyT* kout;
    uint32_t* vout;
    const uint32_t* digit_base;  // [bins] exclusive digit prefix inside the segment
    uint32_t tile;               // global tile index (status row)
    uint32_t first_tile;         // first tile of the segment
    uint32_t tile_n;             // keys in this tile
    uint32_t seg_n;              // keys in the segment
    KeyT key_lo;                 // subtracted from every key before its digit is taken
};

// The last step of a tile: every staged key (and value) to its place.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, bool FULL, bool XF, typename DigitOp>
__device__ __forceinline__ void scatter_staged(const PassParams<DigitOp>& p, const DigitOp& op,
                                               const PassSmem<KeyT>& sm, const TileCtx<KeyT>& c) {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t idx = j * BLOCK + threadIdx.x;
        if (FULL || idx < c.tile_n) {
            const KeyT key = sm.keys[idx];
            const uint32_t d = DigitOp::kStageDigit ? (uint32_t)sm.digs[idx] : op((KeyT)(key - c.key_lo));
            const uint32_t pos = sm.delta[d] + idx;
            if (pos < c.seg_n) {
                c.kout[pos] = XF ? p.xf.from_ordered(key) : key;
                if (VALS) c.vout[pos] = sm.vals[idx];
            }
        }
    }
}

// The body of the pass for one tile; FULL tiles skip every bounds check.
// XF: compiled with the typed-key mapping (p.xf_in / p.xf_out are honoured);
// plain kernels are compiled without it and carry none of its code.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, bool FULL, typename DigitOp, bool XF = false>
__device__ __forceinline__ void onesweep_tile(const PassParams<DigitOp>& p, const DigitOp& op,
                                              const PassSmem<KeyT>& sm, const TileCtx<KeyT>& c, uint32_t bins,
                                              bool publish) {
    constexpr int kSubs = BLOCK / 16;
    constexpr int kTile = BLOCK * ITEMS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const bool first = c.tile == c.first_tile;

    // load: half-warp h of warp w (sub 2w + h) owns the 16*ITEMS keys from
    // (2w + h)*16*ITEMS of the tile; its lane l holds item i = key
    // (2w + h)*16*ITEMS + i*16 + l.  Every load instruction of a warp reads
    // two runs of 16 consecutive keys, one per half.
    const uint32_t hofs = (uint32_t)warp * (ITEMS * 32) + (uint32_t)half * (ITEMS * 16) + hl;
    KeyT k[ITEMS];
    uint32_t v[VALS ? ITEMS : 1];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t idx = hofs + i * 16;
        const bool ok = FULL || idx < c.tile_n;
        k[i] = ok ? c.kin[idx] : c.key_lo;
        if (VALS) v[i] = ok ? c.vin[idx] : 0u;
    }
    if (XF && p.xf_in) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) k[i] = p.xf.to_ordered(k[i]);
    }

    // rank every key inside its half-warp; keep (digit << 16 | rank) per item
    const uint32_t tab = smem_addr(sm.tab + (size_t)(2 * warp + half) * sm.tab_stride);
    const uint32_t hbit = 1u << hl;
    const uint32_t hlt = hbit - 1u;
    const uint32_t hgt = 0xffffu & ~(hlt | hbit);
    // Per item, the digit and rank (digit << 16 | rank).  For digits that
    // are cheap to recompute (plain radix digits) only the 16-bit ranks are
    // kept, two per register, and the digit is taken again from the key
    // when it is staged: 18 registers instead of 36 for 36 keys per thread.
    constexpr bool kPackRanks = !DigitOp::kStageDigit;
    uint32_t dr[kPackRanks ? (ITEMS + 1) / 2 : ITEMS] = {};  // (every word is set before it is read)
    auto put = [&](int i, uint32_t d, uint32_t rank) {
        if (kPackRanks) {
            if (i & 1)
                dr[i >> 1] |= rank << 16;
            else
                dr[i >> 1] = rank;
        } else {
            dr[i] = (d << 16) | rank;
        }
    };
    // A warp whose keys all carry one digit (a run of sorted keys) needs no
    // ranking: a key's rank is its position in its half-warp, and each
    // half-warp's count of that digit is all its keys.  This spares the
    // atomics on one table word that such a warp would make per item.  Full
    // tiles only; screened by the warp's first and last keys (lane 0's first
    // item and lane 31's last), then decided on the warp's smallest and
    // largest keys.
    bool uniform = false;
    if (FULL) {
        const KeyT first = __shfl_sync(0xffffffffu, k[0], 0);
        const KeyT last = __shfl_sync(0xffffffffu, k[ITEMS - 1], 31);
        if (op.same_digit_range((KeyT)(first - c.key_lo), (KeyT)(last - c.key_lo))) {
            KeyT lo = k[0], hi = k[0];
#pragma unroll
            for (int i = 1; i < ITEMS; ++i) {
                lo = k[i] < lo ? k[i] : lo;
                hi = k[i] > hi ? k[i] : hi;
            }
            uniform = op.same_digit_range((KeyT)(warp_min(lo) - c.key_lo), (KeyT)(warp_max(hi) - c.key_lo));
        }
    }
    if (uniform) {
        const uint32_t d0 = op((KeyT)(k[0] - c.key_lo));
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) put(i, d0, (uint32_t)(i * 16 + hl));
        st_shared_u32_if(tab + 4u * d0, (uint32_t)(ITEMS * 16) << 16, hl == 0);
    } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const bool ok = FULL || (hofs + i * 16) < c.tile_n;
            const uint32_t d = op((KeyT)(k[i] - c.key_lo));
            put(i, d, subwarp_rank<FULL>(tab, d, ok, hbit, hlt, hgt));
        }
    }
    __syncthreads();

    // per digit: tile count, publish it, then the look-back right away, so
    // this tile's inclusive prefix is published as early as possible; then
    // each digit's start inside the staged tile, and each half-warp's offset
    // inside that digit (it replaces the rank-table entry)
    uint32_t* srow = p.status + (size_t)c.tile * bins;
    // One digit per thread: its count, look-back and place in the tile's
    // scan stay in registers (two barriers instead of five).  Measured at
    // 100M keys: bucket partition passes 0.535 -> 0.521 ms, u32 key-value
    // sorts 2.398 -> 2.367 ms; but u32 keys alone 0.353 -> 0.358 ms per
    // pass, which keep the path through shared memory.
    constexpr bool kFused = DigitOp::kStageDigit || VALS;
    if (kFused && bins == (uint32_t)BLOCK) {
        const uint32_t d = (uint32_t)tid;
        uint32_t sum = 0;
#pragma unroll
        for (int s = 0; s < kSubs; ++s) sum += sm.tab[(size_t)s * sm.tab_stride + d] >> 16;
        if (publish) st_relaxed(srow + d, (first ? kFlagPrefix : kFlagAggregate) | sum);
        const uint32_t excl =
            first ? 0u : lookback_digit(p.status, c.tile, c.first_tile, bins, d, p.spin_limit, p.hdr);
        if (!first && publish) st_relaxed(srow + d, kFlagPrefix | ((excl + sum) & kCountMask));
        uint32_t run = block_exclusive_sum<BLOCK, false>(sum, sm.scan);
        sm.delta[d] = c.digit_base[d] + excl - run;
#pragma unroll
        for (int s = 0; s < kSubs; ++s) {
            uint32_t* e = sm.tab + (size_t)s * sm.tab_stride + d;
            const uint32_t cnt = *e >> 16;
            *e = run;
            run += cnt;
        }
    } else {
        for (uint32_t d = tid; d < bins; d += BLOCK) {
            uint32_t sum = 0;
#pragma unroll
            for (int s = 0; s < kSubs; ++s) sum += sm.tab[(size_t)s * sm.tab_stride + d] >> 16;
            sm.local[d] = sum;
            if (publish) st_relaxed(srow + d, (first ? kFlagPrefix : kFlagAggregate) | sum);
        }
        for (uint32_t d = tid; d < bins; d += BLOCK) {
            const uint32_t excl =
                first ? 0u : lookback_digit(p.status, c.tile, c.first_tile, bins, d, p.spin_limit, p.hdr);
            if (!first && publish) st_relaxed(srow + d, kFlagPrefix | ((excl + sm.local[d]) & kCountMask));
            sm.delta[d] = c.digit_base[d] + excl;
        }
        __syncthreads();
        block_exclusive_scan_smem<BLOCK>(sm.local, (int)bins, sm.scan);
        for (uint32_t d = tid; d < bins; d += BLOCK) {
            uint32_t run = sm.local[d];
            sm.delta[d] -= run;
#pragma unroll
            for (int s = 0; s < kSubs; ++s) {
                uint32_t* e = sm.tab + (size_t)s * sm.tab_stride + d;
                const uint32_t cnt = *e >> 16;
                *e = run;
                run += cnt;
            }
        }
    }
    __syncthreads();

    // stage the tile in shared memory in digit order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = FULL || (hofs + i * 16) < c.tile_n;
        if (ok) {
            const uint32_t d = kPackRanks ? op((KeyT)(k[i] - c.key_lo)) : (dr[i] >> 16);
            const uint32_t rank = kPackRanks ? ((dr[i >> 1] >> (16 * (i & 1))) & 0xffffu) : (dr[i] & 0xffffu);
            const uint32_t pos = ld_shared_u32(tab + 4u * d) + rank;
            if (pos < (uint32_t)kTile) {
                sm.keys[pos] = k[i];
                if (VALS) sm.vals[pos] = v[i];
                if (DigitOp::kStageDigit) sm.digs[pos] = (uint8_t)d;
            }
        }
    }
    __syncthreads();

    // write runs of equal digits to their places in the segment (typed keys
    // are mapped back in a separate copy of the loop)
    if (XF && p.xf_out)
        scatter_staged<KeyT, VALS, BLOCK, ITEMS, FULL, true>(p, op, sm, c);
    else
        scatter_staged<KeyT, VALS, BLOCK, ITEMS, FULL, false>(p, op, sm, c);
}

// A pass whose keys all carry one digit: the counting sort leaves their
// order unchanged (Algorithm 3 places the keys of one digit in input order),
// so the pass is a copy of its input, with the typed-key mapping of its place
// in the sort.  The status words of the next pass are still cleared.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, typename DigitOp, bool XF>
__device__ __forceinline__ void identity_pass(const PassParams<DigitOp>& p, uint32_t bins) {
    constexpr uint32_t kTile = BLOCK * ITEMS;
    const KeyT* kin = static_cast<const KeyT*>(p.keys_in);
    KeyT* kout = static_cast<KeyT*>(p.keys_out);
    for (uint32_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
        if (p.status_next)
            for (uint32_t d = threadIdx.x; d < bins; d += BLOCK) p.status_next[(size_t)tile * bins + d] = 0u;
        const uint32_t base = tile * kTile;
        const uint32_t m = min(kTile, p.n - base);
        KeyT k[ITEMS];
        uint32_t v[VALS ? ITEMS : 1];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t idx = i * BLOCK + threadIdx.x;
            k[i] = idx < m ? kin[base + idx] : (KeyT)0;
            if (VALS) v[i] = idx < m ? p.vals_in[base + idx] : 0u;
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t idx = i * BLOCK + threadIdx.x;
            if (idx < m) {
                KeyT key = k[i];
                if (XF && p.xf_in) key = p.xf.to_ordered(key);
                if (XF && p.xf_out) key = p.xf.from_ordered(key);
                kout[base + idx] = key;
                if (VALS) p.vals_out[base + idx] = v[i];
            }
        }
    }
}

// Ask `count` keys (and values) into L2: one prefetch per 128-byte line,
// spread over the block's threads.
template <typename KeyT, bool VALS, int BLOCK>
__device__ __forceinline__ void prefetch_l2(const KeyT* keys, const uint32_t* vals, size_t count) {
    const char* kb = reinterpret_cast<const char*>(keys);
    const uint32_t klines = (uint32_t)((count * sizeof(KeyT) + 127) / 128);
    for (uint32_t i = threadIdx.x; i < klines; i += BLOCK)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(kb + (size_t)i * 128));
    if (VALS) {
        const char* vb = reinterpret_cast<const char*>(vals);
        const uint32_t vlines = (uint32_t)((count * 4 + 127) / 128);
        for (uint32_t i = threadIdx.x; i < vlines; i += BLOCK)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(vb + (size_t)i * 128));
    }
}

// Persistent: every block claims tiles from the pass's counter until none is
// left.  A block holds one tile at a time and only waits on tiles claimed
// earlier, whose blocks are running, so the waits always end.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB, typename DigitOp, bool XF = false>
__global__ void __launch_bounds__(BLOCK, MINB) k_onesweep(PassParams<DigitOp> p) {
    constexpr int kTile = BLOCK * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tile;
    const uint32_t bins = 1u << p.digit_bits;
    const PassSmem<KeyT> sm = carve_pass_smem<KeyT, VALS, BLOCK>(smem, bins, kTile);
    DigitOp op = p.op;
    op.init();
    const int tid = threadIdx.x;
    // every key carries the first key's digit iff that digit's exclusive
    // prefix is 0 and the next digit's is n
    if (tid == 0) {
        KeyT k0 = static_cast<const KeyT*>(p.keys_in)[0];
        if (XF && p.xf_in) k0 = p.xf.to_ordered(k0);
        const uint32_t d0 = op(k0);
        s_tile = p.digit_base[d0] == 0u && (d0 + 1u == bins || p.digit_base[d0 + 1u] == p.n);
    }
    __syncthreads();
    if (s_tile) {
        identity_pass<KeyT, VALS, BLOCK, ITEMS, DigitOp, XF>(p, bins);
        return;
    }
    __syncthreads();  // s_tile is reused for the tile ids below
    while (true) {
        for (uint32_t i = tid; i < (uint32_t)(BLOCK / 16) * sm.tab_stride; i += BLOCK) sm.tab[i] = 0u;
        if (tid == 0) s_tile = atomicAdd(p.tile_ctr, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= p.num_tiles) return;  // uniform across the block
        if (p.status_next)
            for (uint32_t d = tid; d < bins; d += BLOCK) p.status_next[(size_t)tile * bins + d] = 0u;
        // Tiles are claimed in order, so the tile one grid ahead is about
        // the one this block takes next: its keys (and values) are asked
        // into L2 now, one 128-byte line per thread, and its loads then
        // wait on L2 rather than on DRAM.  Measured at 100M keys: u64 keys
        // with values 0.787 -> 0.764 ms per pass, 40-bit u64 keys 0.293 ->
        // 0.286; u32 keys alone 0.353 -> 0.356, so not for 4-byte items,
        // and no gain for the bucket sort's partition passes (bound by their
        // digits), nor in the segmented pass.
        constexpr bool kPrefetch = !DigitOp::kStageDigit && sizeof(KeyT) + (VALS ? 4 : 0) >= 8;
        if (kPrefetch && tile + gridDim.x < p.num_tiles) {
            const size_t first = (size_t)(tile + gridDim.x) * kTile;
            prefetch_l2<KeyT, VALS, BLOCK>(static_cast<const KeyT*>(p.keys_in) + first,
                                           VALS ? p.vals_in + first : nullptr,
                                           min((size_t)kTile, (size_t)p.n - first));
        }
        TileCtx<KeyT> c;
        const uint32_t base = tile * (uint32_t)kTile;
        c.kin = static_cast<const KeyT*>(p.keys_in) + base;
        c.vin = VALS ? p.vals_in + base : nullptr;
        c.kout = static_cast<KeyT*>(p.keys_out);
        c.vout = p.vals_out;
        c.digit_base = p.digit_base;
        c.tile = tile;
        c.first_tile = 0;
        c.tile_n = min((uint32_t)kTile, p.n - base);
        c.seg_n = p.n;
        c.key_lo = 0;
        const bool publish = (int)tile != p.stall_tile;
        if (c.tile_n == (uint32_t)kTile)
            onesweep_tile<KeyT, VALS, BLOCK, ITEMS, true, DigitOp, XF>(p, op, sm, c, bins, publish);
        else
            onesweep_tile<KeyT, VALS, BLOCK, ITEMS, false, DigitOp, XF>(p, op, sm, c, bins, publish);
        __syncthreads();
    }
}

// Checked mode: every key of a sort's output is at most the next one in the
// sort's order (typed keys compared by their ordered image); the first pair
// out of order is recorded as RS_ERR_CHECK_FAILED.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_check_order(const KeyT* __restrict__ keys, size_t n, KeyXform xf,
                                                     WsHeader* hdr) {
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i + 1 < n; i += (size_t)gridDim.x * 256) {
        if (xf.to_ordered(keys[i + 1]) < xf.to_ordered(keys[i])) {
            set_device_error(hdr, RS_ERR_CHECK_FAILED, (uint32_t)i);
            return;
        }
    }
}

// Blocks of a kernel that fit on the GPU at once (the grid of a persistent
// launch); at least 1.  The occupancy query is cached per (kernel, shared
// memory, device): it costs host time on every launch otherwise.
int resident_grid_cached(const void* kern, int block, size_t smem, int (*query)(const void*, int, size_t));

template <typename Kernel>
int resident_grid(Kernel kern, int block, size_t smem) {
    return resident_grid_cached(
        reinterpret_cast<const void*>(kern), block, smem, [](const void* k, int b, size_t sm) -> int {
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<Kernel>(const_cast<void*>(k)),
                                                              b, sm) != cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            return per_sm;
        });
}

}  // namespace rs
