// rs_bucket.cuh -- the bucket function of the bucket sort (Sec. 2.3,
// Algorithm 2) on the device, and the digit views of it that the counting,
// scatter and shared-memory kernels use.
//
// The bucket of key k among nb buckets covering [min, max] is
//     b(k) = floor((k - min) * nb / (max - min + 1)),
// computed exactly: it is the paper's n * A[i] / M with the key range made
// inclusive and kept inside [0, nb - 1].  b is nondecreasing in k, so sorting
// by (bucket, key) is sorting by key.
#pragma once

#include "rs_segmented.cuh"

namespace rs {

struct BucketParams {
    uint64_t min;    // lowest key of the range
    uint64_t max;    // highest key of the range
    uint64_t nb;     // number of buckets
    uint64_t range;  // max - min + 1; 0 stands for 2^64
    uint64_t recip;  // floor((2^64 - 1) / range) when range <= 2^32
    uint64_t mul;    // floor(2^64 * nb / range) when nb < range (mul_ok)
    uint32_t bbits;  // bit length of nb - 1 (0 when nb == 1)
    uint32_t valid;  // 1 once the parameters are set
    uint32_t mul_ok;
    uint32_t pad;
};

// Exact floor((k - min) * nb / range).
//   32-bit keys: x = (k - min) * nb < 2^64 and range <= 2^32; the estimate
//   q = mulhi(x, floor((2^64-1)/range)) is at most 2 below the quotient
//   (division by an invariant integer through a precomputed reciprocal,
//   Granlund & Montgomery 1994), and the remainder test corrects it.
//   64-bit keys with nb < range: the same estimate with 64-bit words,
//   m = floor(2^64 nb / range) and e = floor(u m / 2^64) (a 64 x 64 high
//   product), is the quotient or one below it for the same reason, and the
//   exact comparison (e + 1) * range <= u * nb is made on 128-bit products
//   (multiplications only; no division per key).  64-bit keys with
//   nb >= range have range <= 2^32 and u * nb < 2^64, so they take the
//   32-bit keys' reciprocal path; range 2^64 is a plain high product.
//   32-bit keys with nb < range take a cheaper estimate first: with
//   m = floor(2^64 nb / range), e = floor(t m / 2^64) (t = k - min, a 32 x 64
//   bit high product) is the quotient or one below it (m is short of
//   2^64 nb / range by less than 1 and t < 2^32), and one exact comparison
//   (e + 1) * range <= t * nb settles which.
__device__ __forceinline__ uint64_t bucket_of(const BucketParams& bp, uint32_t k) {
    const uint32_t t = k - (uint32_t)bp.min;
    if (bp.mul_ok) {
        // nb < range <= 2^32, so the estimate e <= floor(t nb / range) < nb
        // and e + 1 fit 32 bits, and both sides of the exact comparison are
        // sums of 32 x 32-bit products (range split into its low word and
        // bit 32): no 64 x 64-bit multiplication per key
        const uint32_t e =
            (uint32_t)(((uint64_t)t * (uint32_t)(bp.mul >> 32) + __umulhi(t, (uint32_t)bp.mul)) >> 32);
        const uint64_t lhs =
            (uint64_t)(e + 1u) * (uint32_t)bp.range + ((bp.range >> 32) ? ((uint64_t)(e + 1u) << 32) : 0ull);
        return (uint64_t)(e + (uint32_t)(lhs <= (uint64_t)t * (uint32_t)bp.nb));
    }
    const uint64_t x = (uint64_t)t * bp.nb;
    uint64_t q = __umul64hi(x, bp.recip);
    uint64_t r = x - q * bp.range;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        if (r >= bp.range) {
            ++q;
            r -= bp.range;
        }
    return q;
}

__device__ __forceinline__ uint64_t bucket_of(const BucketParams& bp, uint64_t k) {
    const uint64_t u = k - bp.min;
    if (bp.range == 0) return __umul64hi(u, bp.nb);
    if (bp.mul_ok) {
        const uint64_t e = __umul64hi(u, bp.mul);
        const unsigned __int128 lhs = (unsigned __int128)(e + 1) * bp.range;
        const unsigned __int128 rhs = (unsigned __int128)u * bp.nb;
        return e + (uint64_t)(lhs <= rhs);
    }
    const uint64_t x = u * bp.nb;  // < 2^64: range <= 2^32 here
    uint64_t q = __umul64hi(x, bp.recip);
    uint64_t r = x - q * bp.range;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        if (r >= bp.range) {
            ++q;
            r -= bp.range;
        }
    return q;
}

// min <= k <= max; for 32-bit keys max - min < 2^32, so one 32-bit
// subtraction and comparison decide it.
__device__ __forceinline__ bool key_in_bounds(const BucketParams& bp, uint32_t k) {
    return k - (uint32_t)bp.min <= (uint32_t)(bp.max - bp.min);
}
__device__ __forceinline__ bool key_in_bounds(const BucketParams& bp, uint64_t k) {
    return k >= bp.min && k <= bp.max;
}

__device__ __forceinline__ BucketParams load_bucket_params(const BucketParams* p) {
    BucketParams b;
    b.min = __ldcg(&p->min);
    b.max = __ldcg(&p->max);
    b.nb = __ldcg(&p->nb);
    b.range = __ldcg(&p->range);
    b.recip = __ldcg(&p->recip);
    b.mul = __ldcg(&p->mul);
    b.bbits = __ldcg(&p->bbits);
    b.valid = __ldcg(&p->valid);
    b.mul_ok = __ldcg(&p->mul_ok);
    b.pad = 0;
    return b;
}

// Position (shift) and width (bits) of the bucket-id digit that partition
// level 1 or 2 sorts by, for a bucket id of bbits bits: level 1 takes the top
// min(8, bbits) bits, level 2 the next min(8, what is left) bits.
__host__ __device__ __forceinline__ void bucket_level_digit(uint32_t bbits, int level, int* shift, int* bits) {
    const int d1 = bbits < 8u ? (int)bbits : 8;
    const int s1 = (int)bbits - d1;
    if (level <= 1) {
        *shift = s1;
        *bits = d1;
    } else {
        const int d2 = s1 < 8 ? s1 : 8;
        *shift = s1 - d2;
        *bits = d2;
    }
}

// Digit of the bucket id for a scatter pass: (b(k) >> shift) & mask.  With a
// table (the segmented bucket sort), every segment has its own parameters
// (table[SegDesc::grp]) and the digit is that of partition level `level` for
// the segment's bucket-id width; for_segment selects them per tile.
struct BucketDigit {
    static constexpr bool kStageDigit = true;  // a bucket id costs more than a staged byte: stage it
    const BucketParams* src;
    int shift;
    uint32_t mask;
    BucketParams bp;
    const BucketParams* table = nullptr;
    int level = 0;
    __device__ __forceinline__ void init() {
        if (!table) bp = load_bucket_params(src);
    }
    template <typename Seg>
    __device__ __forceinline__ void for_segment(const Seg& s) {
        if (!table) return;
        bp = load_bucket_params(table + s.grp);
        int bits;
        bucket_level_digit(bp.bbits, level, &shift, &bits);
        mask = (1u << bits) - 1u;
    }
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT k) const {
        return (uint32_t)(bucket_of(bp, k) >> shift) & mask;
    }
    // every key in [lo, hi] has one digit (the bucket id is monotone in the key)
    template <typename KeyT>
    __device__ __forceinline__ bool same_digit_range(KeyT lo, KeyT hi) const {
        return (bucket_of(bp, lo) >> shift) == (bucket_of(bp, hi) >> shift);
    }
};

// The same digit for the counting kernels (only pass q = 0 exists).  With
// check_range, keys outside the segment's [min, max] are reported (declared
// bounds of the segmented bucket sort).
struct BucketDigits {
    static constexpr bool kBytesCapable = false;
    static constexpr bool kOneDigit = true;
    const BucketParams* src;
    int shift;
    uint32_t mask;
    BucketParams bp;
    const BucketParams* table = nullptr;
    int level = 0;
    int check_range = 0;
    __device__ __forceinline__ void init() {
        if (!table) bp = load_bucket_params(src);
    }
    template <typename Seg>
    __device__ __forceinline__ void for_segment(const Seg& s) {
        if (!table) return;
        bp = load_bucket_params(table + s.grp);
        int bits;
        bucket_level_digit(bp.bbits, level, &shift, &bits);
        mask = (1u << bits) - 1u;
    }
    template <typename KeyT>
    __device__ __forceinline__ uint32_t operator()(KeyT k, int) const {
        return (uint32_t)(bucket_of(bp, k) >> shift) & mask;
    }
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT k) const {
        return !check_range || key_in_bounds(bp, k);
    }
    __device__ __forceinline__ bool byte_digits() const { return false; }
};

// Bucket view for the shared-memory sort of one partition: the partition's
// first bucket is kept in SegDesc::aux and the number of buckets it spans in
// SegDesc::chunk0 (unused for shared-memory segments).
// With a table (the segmented bucket sort), each segment's parameters are
// table[SegDesc::grp], and with check_range its keys must lie in [min, max].
struct SegBucketFn {
    const BucketParams* src;
    BucketParams bp;
    const BucketParams* table = nullptr;
    int check_range = 0;
    __device__ __forceinline__ bool active() const { return src != nullptr || table != nullptr; }
    __device__ __forceinline__ void init() {
        if (!table) bp = load_bucket_params(src);
    }
    __device__ __forceinline__ void for_segment(const SegDesc& s) {
        if (table) bp = load_bucket_params(table + s.grp);
    }
    template <typename KeyT>
    __device__ __forceinline__ bool in_range(KeyT k) const {
        return !check_range || key_in_bounds(bp, k);
    }
    __device__ __forceinline__ uint64_t first_bucket(const SegDesc& s) const { return s.aux; }
    __device__ __forceinline__ uint64_t bucket_span(const SegDesc& s) const { return s.chunk0; }
    template <typename KeyT>
    __device__ __forceinline__ uint64_t bucket(KeyT k) const {
        return bucket_of(bp, k);
    }
};

}  // namespace rs
