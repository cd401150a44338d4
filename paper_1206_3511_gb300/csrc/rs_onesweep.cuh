// rs_onesweep.cuh -- the two kernels of one LSD radix sort on the GPU.
//
//  k_digit_counts: the counting loop of the counting sort (Sec. 2.4,
//    Algorithm 3) for every pass of the radix sort (Sec. 2.5, Algorithm 4) in
//    one read of the keys; the last block turns the counts into exclusive
//    prefixes, which are the counting sort's "number of smaller digits".
//
//  k_onesweep: one stable counting-sort pass (the placement loop of Algorithm
//    3) done block-wise: each block takes the next tile (dynamic tile id),
//    ranks its keys stably by digit in shared memory (warp multisplit with
//    __match_any_sync, Adinets & Merrill, "Onesweep", arXiv:2206.01784),
//    obtains the number of equal digits in all earlier tiles through a
//    decoupled look-back over per-(tile, digit) status words, and writes each
//    key to  digit_base[d] + (earlier tiles' d) + (rank inside the tile).
//    The keys are read once and written once per pass.
#pragma once

#include "rs_common.cuh"

namespace rs {

// Digit of a key for plain LSD radix sort: (key >> shift) & mask.
struct RadixDigit {
    int shift;
    uint32_t mask;
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT k) const {
        return (uint32_t)(k >> shift) & mask;
    }
};

// ---------------------------------------------------------------------------
// Digit counts of every pass in one read.
struct CountParams {
    const void* keys;
    size_t n;
    int shift0;      // digit p is (key >> (shift0 + p*D)) & (2^D - 1)
    int digit_bits;  // D
    int passes;      // P
    int key_bits;    // keys must be < 2^key_bits; >= key width disables the check
    uint32_t* counts;  // [P][2^D], zero on entry
    uint32_t* scan;    // [P][2^D] exclusive prefixes (nullable)
    uint32_t* zero_ptr;  // words zeroed by the kernel (first pass's status words)
    size_t zero_words;
    WsHeader* hdr;
};

constexpr int kCountBlock = 512;
constexpr int kCountItems = 16;

template <typename KeyT>
__global__ void __launch_bounds__(kCountBlock) k_digit_counts(CountParams p) {
    extern __shared__ uint32_t s_cnt[];  // [P][bins], then kCountBlock/32+1 scan words
    __shared__ uint32_t s_last;
    const uint32_t bins = 1u << p.digit_bits, mask = bins - 1u;
    const int ncnt = p.passes * (int)bins;
    uint32_t* s_scan = s_cnt + ncnt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < ncnt; i += kCountBlock) s_cnt[i] = 0;
    for (size_t i = (size_t)blockIdx.x * kCountBlock + tid; i < p.zero_words; i += (size_t)gridDim.x * kCountBlock)
        p.zero_ptr[i] = 0;
    __syncthreads();

    const KeyT* keys = static_cast<const KeyT*>(p.keys);
    constexpr size_t kChunk = (size_t)kCountBlock * kCountItems;
    KeyT seen = 0;
    for (size_t base = (size_t)blockIdx.x * kChunk; base < p.n; base += (size_t)gridDim.x * kChunk) {
        const size_t wbase = base + (size_t)warp * (32 * kCountItems) + lane;
        const bool full = base + kChunk <= p.n;
        KeyT k[kCountItems];
#pragma unroll
        for (int i = 0; i < kCountItems; ++i) {
            size_t idx = wbase + (size_t)i * 32;
            k[i] = (full || idx < p.n) ? __ldcs(keys + idx) : (KeyT)0;
        }
#pragma unroll
        for (int i = 0; i < kCountItems; ++i) {
            const bool valid = full || (wbase + (size_t)i * 32 < p.n);
            if (valid) seen |= k[i];
            for (int q = 0; q < p.passes; ++q) {
                const uint32_t d = (uint32_t)(k[i] >> (p.shift0 + q * p.digit_bits)) & mask;
                // all 32 lanes on one digit (sorted or narrow-range input):
                // one shared atomic instead of 32 conflicting ones
                const uint32_t d0 = __shfl_sync(kFullMask, d, 0);
                if (__all_sync(kFullMask, valid && d == d0)) {
                    if (lane == 0) atomicAdd(&s_cnt[q * bins + d], 32u);
                } else if (valid) {
                    atomicAdd(&s_cnt[q * bins + d], 1u);
                }
            }
        }
    }
    if (p.key_bits < (int)(8 * sizeof(KeyT)) && (seen >> p.key_bits) != 0)
        set_device_error(p.hdr, RS_ERR_KEY_RANGE, blockIdx.x);
    __syncthreads();
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
    for (int q = 0; q < p.passes; ++q) {
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
};

template <typename KeyT, bool VALS, int BLOCK, int ITEMS>
struct OnesweepShape {
    static constexpr int kWarps = BLOCK / 32;
    static constexpr int kTile = BLOCK * ITEMS;
    static_assert(kTile < 65536, "per-warp counters are 16-bit");
    static size_t smem_bytes(int digit_bits) {
        const size_t bins = (size_t)1 << digit_bits;
        size_t b = (size_t)kTile * sizeof(KeyT);
        if (VALS) b += (size_t)kTile * 4;
        b += align_up((size_t)kWarps * bins * 2, 16);  // per-warp digit counters (u16)
        b += bins * 4 * 3;                             // tile counts, local starts, scatter deltas
        b += (kWarps + 1 + 3) * 4;                     // scan scratch, tile id
        return b;
    }
};

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, typename DigitOp>
__global__ void __launch_bounds__(BLOCK) k_onesweep(PassParams<DigitOp> p) {
    using Shape = OnesweepShape<KeyT, VALS, BLOCK, ITEMS>;
    constexpr int kWarps = Shape::kWarps;
    constexpr int kTile = Shape::kTile;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t bins = 1u << p.digit_bits;
    KeyT* s_keys = reinterpret_cast<KeyT*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kTile);
    uint16_t* s_wcnt = reinterpret_cast<uint16_t*>(s_vals + (VALS ? kTile : 0));
    uint32_t* s_tcnt = reinterpret_cast<uint32_t*>(
        reinterpret_cast<unsigned char*>(s_wcnt) + align_up((size_t)kWarps * bins * 2, 16));
    uint32_t* s_local = s_tcnt + bins;
    uint32_t* s_delta = s_local + bins;
    uint32_t* s_scan = s_delta + bins;  // kWarps + 1 words
    uint32_t* s_tile = s_scan + kWarps + 1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t i = tid; i < (uint32_t)kWarps * bins; i += BLOCK) s_wcnt[i] = 0;
    if (tid == 0) *s_tile = atomicAdd(p.tile_ctr, 1u);
    __syncthreads();
    const uint32_t tile = *s_tile;
    if (tile >= p.num_tiles) return;  // uniform across the block
    const bool publish = (int)tile != p.stall_tile;
    if (p.status_next)
        for (uint32_t d = tid; d < bins; d += BLOCK) p.status_next[(size_t)tile * bins + d] = 0u;

    const uint32_t tile_base = tile * (uint32_t)kTile;
    const uint32_t tile_n = min((uint32_t)kTile, p.n - tile_base);
    const bool full = tile_n == (uint32_t)kTile;

    // load: warp w owns keys [w*ITEMS*32, (w+1)*ITEMS*32) of the tile, lane l
    // holds item i = key w*ITEMS*32 + i*32 + l (warp-striped, coalesced)
    const KeyT* kin = static_cast<const KeyT*>(p.keys_in) + tile_base;
    const uint32_t wofs = (uint32_t)warp * (ITEMS * 32) + lane;
    KeyT k[ITEMS];
    uint32_t v[VALS ? ITEMS : 1];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t idx = wofs + i * 32;
        const bool ok = full || idx < tile_n;
        k[i] = ok ? kin[idx] : (KeyT)0;
        if (VALS) v[i] = ok ? p.vals_in[tile_base + idx] : 0u;
    }

    // stable rank inside the warp: lanes with equal digits form one peer
    // group; the group's last lane bumps the warp's counter for that digit
    uint16_t* wc = s_wcnt + warp * bins;
    uint32_t rank[ITEMS];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = full || (wofs + i * 32) < tile_n;
        const uint32_t d = ok ? p.op(k[i]) : bins;  // padding lanes group apart
        const uint32_t peers = __match_any_sync(kFullMask, d);
        const int leader = 31 - __clz(peers);
        uint32_t before = 0;
        if (lane == leader && ok) {
            before = wc[d];
            wc[d] = (uint16_t)(before + __popc(peers));
        }
        before = __shfl_sync(kFullMask, before, leader);
        rank[i] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();

    // per digit: warp-exclusive prefixes, tile count, publish the count
    uint32_t* srow = p.status + (size_t)tile * bins;
    for (uint32_t d = tid; d < bins; d += BLOCK) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = s_wcnt[w * bins + d];
            s_wcnt[w * bins + d] = (uint16_t)sum;
            sum += c;
        }
        s_tcnt[d] = sum;
        s_local[d] = sum;
        if (publish) st_relaxed(srow + d, (tile == 0 ? kFlagPrefix : kFlagAggregate) | sum);
    }
    __syncthreads();
    block_exclusive_scan_smem<BLOCK>(s_local, (int)bins, s_scan);

    // stage the tile in shared memory in digit order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const bool ok = full || (wofs + i * 32) < tile_n;
        if (ok) {
            const uint32_t d = p.op(k[i]);
            const uint32_t pos = s_local[d] + wc[d] + rank[i];
            if (pos < (uint32_t)kTile) {
                s_keys[pos] = k[i];
                if (VALS) s_vals[pos] = v[i];
            }
        }
    }

    // decoupled look-back: count of digit d in all earlier tiles
    for (uint32_t d = tid; d < bins; d += BLOCK) {
        uint32_t excl = 0;
        if (tile != 0) {
            int t = (int)tile - 1;
            uint32_t polls = 0;
            while (true) {
                const uint32_t s = ld_relaxed(p.status + (size_t)t * bins + d);
                const uint32_t flag = s & ~kCountMask;
                if (flag == kFlagInvalid) {
                    if (++polls > p.spin_limit) {
                        set_device_error(p.hdr, RS_ERR_DEVICE_TIMEOUT, tile);
                        break;  // partial prefix <= true prefix: writes stay in bounds
                    }
                    if (polls > 16) __nanosleep(polls < 256 ? 64 : 512);
                    continue;
                }
                excl += s & kCountMask;
                if (flag == kFlagPrefix || t == 0) break;
                --t;
            }
            if (publish) st_relaxed(srow + d, kFlagPrefix | ((excl + s_tcnt[d]) & kCountMask));
        }
        s_delta[d] = p.digit_base[d] + excl - s_local[d];
    }
    __syncthreads();

    // write runs of equal digits to their global places
    KeyT* kout = static_cast<KeyT*>(p.keys_out);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t idx = j * BLOCK + tid;
        if (full || idx < tile_n) {
            const KeyT key = s_keys[idx];
            const uint32_t pos = s_delta[p.op(key)] + idx;
            if (pos < p.n) {
                kout[pos] = key;
                if (VALS) p.vals_out[pos] = s_vals[idx];
            }
        }
    }
}

}  // namespace rs
