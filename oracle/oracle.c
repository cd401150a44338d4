/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the two integer
 * sorts of Horsmalahti, "Comparison of Bucket Sort and RADIX Sort"
 * (arXiv:1206.3511).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the GPU library is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Every routine follows the paper's definitions in the paper's order, with
 * 0-based arrays:
 *   - the problem (Sec. 2): output a nondecreasing permutation of the input;
 *     a sort is stable when equal keys keep their input order;
 *   - INSERTION-SORT (Sec. 2.2, Algorithm 1);
 *   - BUCKET-SORT (Sec. 2.3, Algorithm 2);
 *   - COUNTING-SORT (Sec. 2.4, Algorithm 3);
 *   - RADIX-SORT, least significant digit first (Sec. 2.5, Algorithm 4).
 *
 * Keys are unsigned 64-bit integers; 32-bit keys are widened by the caller.
 * An optional 32-bit payload ("value") moves with each key.  All arithmetic is
 * integer.  Readings of the paper where it is silent or inconsistent:
 *   R1  digits are D-bit binary digits, digit p of k = (k >> pD) & (2^D - 1);
 *       the paper does not fix the base (Sec. 2.5 "e.g. 0...9").
 *   R2  the counting sort keeps 2^D counters and places elements with an
 *       exclusive prefix and a forward loop.  The paper's form (Algorithm 3:
 *       inclusive prefix, backward loop) yields the same stable permutation;
 *       both are here and a test checks that they agree.
 *   R3  the bucket of key k is floor((k - min) * nb / (max - min + 1)),
 *       computed exactly in 128-bit arithmetic.  It is the paper's
 *       n * A[i] / M (Sec. 2.3) with the key range made inclusive, the bucket
 *       count nb a parameter, and the index kept inside [0, nb - 1].
 *   R4  keys enter their bucket at the tail, in input order ("equal keys are
 *       inserted in order", Sec. 2.3), so bucket sort is stable.
 *   R5  the number of passes is ceil(key_bits / D) ("at most d digits",
 *       Sec. 2.5); every key must be below 2^key_bits.
 *
 * Return codes: 0 success, -1 bad argument, -2 key out of the declared range,
 * -3 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORACLE_OK 0
#define ORACLE_EARG -1
#define ORACLE_ERANGE -2
#define ORACLE_ENOMEM -3

static uint64_t digit_of(uint64_t key, int shift, int digit_bits)
{
    uint64_t mask = (digit_bits >= 64) ? ~0ull : ((1ull << digit_bits) - 1ull);
    return shift >= 64 ? 0 : ((key >> shift) & mask);
}

/* ---------------------------------------------------------------------------
 * Sec. 2.4, Algorithm 3 (COUNTING-SORT) on one digit, reading R2: zero the
 * counters, count each digit value, turn the counts into an exclusive prefix
 * (C[d] = number of elements whose digit is below d), then walk the input
 * forward and place each element at C[digit] before incrementing it.
 * Stable because equal digits are placed in input order.
 */
int oracle_counting_pass_u64(const uint64_t* a, const uint32_t* av, uint64_t* b,
                             uint32_t* bv, size_t n, int shift, int digit_bits)
{
    if (digit_bits < 1 || digit_bits > 20 || shift < 0) return ORACLE_EARG;
    size_t k = (size_t)1 << digit_bits;
    uint64_t* C = (uint64_t*)calloc(k, sizeof(uint64_t));
    if (!C) return ORACLE_ENOMEM;
    for (size_t j = 0; j < n; ++j) C[digit_of(a[j], shift, digit_bits)] += 1;
    uint64_t running = 0;
    for (size_t i = 0; i < k; ++i) {
        uint64_t c = C[i];
        C[i] = running;
        running += c;
    }
    for (size_t j = 0; j < n; ++j) {
        uint64_t d = digit_of(a[j], shift, digit_bits);
        uint64_t pos = C[d];
        C[d] = pos + 1;
        b[pos] = a[j];
        if (av && bv) bv[pos] = av[j];
    }
    free(C);
    return ORACLE_OK;
}

/* Sec. 2.4, Algorithm 3 exactly as printed, shifted to 0-based arrays: the
 * counters become an inclusive prefix (C[d] = number of elements whose digit
 * is at most d) and the final loop walks the input backward, decrementing
 * C[digit] and storing at the decremented slot.  Used only to check reading R2. */
int oracle_counting_pass_backward_u64(const uint64_t* a, const uint32_t* av, uint64_t* b,
                                      uint32_t* bv, size_t n, int shift, int digit_bits)
{
    if (digit_bits < 1 || digit_bits > 20 || shift < 0) return ORACLE_EARG;
    size_t k = (size_t)1 << digit_bits;
    uint64_t* C = (uint64_t*)calloc(k, sizeof(uint64_t));
    if (!C) return ORACLE_ENOMEM;
    for (size_t j = 0; j < n; ++j) C[digit_of(a[j], shift, digit_bits)] += 1;
    for (size_t i = 1; i < k; ++i) C[i] = C[i] + C[i - 1];
    for (size_t j = n; j > 0; --j) {
        uint64_t d = digit_of(a[j - 1], shift, digit_bits);
        C[d] = C[d] - 1;
        b[C[d]] = a[j - 1];
        if (av && bv) bv[C[d]] = av[j - 1];
    }
    free(C);
    return ORACLE_OK;
}

/* Number of digit passes for keys below 2^key_bits (reading R5). */
int oracle_num_passes(int key_bits, int digit_bits)
{
    if (key_bits < 1 || digit_bits < 1) return 0;
    return (key_bits + digit_bits - 1) / digit_bits;
}

static int keys_fit(const uint64_t* keys, size_t n, int key_bits)
{
    if (key_bits >= 64) return 1;
    uint64_t limit = 1ull << key_bits;
    for (size_t i = 0; i < n; ++i)
        if (keys[i] >= limit) return 0;
    return 1;
}

/* Per-digit counts of every pass: counts[p * 2^D + d] = number of keys whose
 * digit p equals d.  These are the counts Algorithm 3 builds in its second
 * loop, for each of the passes of Algorithm 4. */
int oracle_digit_counts_u64(const uint64_t* keys, size_t n, int key_bits, int digit_bits,
                            uint64_t* counts)
{
    if (key_bits < 1 || key_bits > 64 || digit_bits < 1 || digit_bits > 20) return ORACLE_EARG;
    if (!keys_fit(keys, n, key_bits)) return ORACLE_ERANGE;
    int P = oracle_num_passes(key_bits, digit_bits);
    size_t k = (size_t)1 << digit_bits;
    memset(counts, 0, sizeof(uint64_t) * k * (size_t)P);
    for (int p = 0; p < P; ++p)
        for (size_t i = 0; i < n; ++i) counts[(size_t)p * k + digit_of(keys[i], p * digit_bits, digit_bits)] += 1;
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * Sec. 2.5, Algorithm 4 (RADIX-SORT, LSD): for digit 1 (least significant) to
 * d, stable-sort the whole array on that digit with the counting sort above.
 * Optionally stops after `max_passes` passes (the partial result after pass p
 * is the input stably sorted on its low (p+1)*D bits); max_passes < 0 means
 * all passes. */
int oracle_radix_sort_partial_u64(const uint64_t* keys, const uint32_t* vals, size_t n,
                                  int key_bits, int digit_bits, int max_passes,
                                  uint64_t* out_keys, uint32_t* out_vals)
{
    if (key_bits < 1 || key_bits > 64 || digit_bits < 1 || digit_bits > 20) return ORACLE_EARG;
    if (!keys_fit(keys, n, key_bits)) return ORACLE_ERANGE;
    int P = oracle_num_passes(key_bits, digit_bits);
    if (max_passes >= 0 && max_passes < P) P = max_passes;
    size_t nn = n ? n : 1;
    uint64_t* A = (uint64_t*)malloc(nn * sizeof(uint64_t));
    uint64_t* B = (uint64_t*)malloc(nn * sizeof(uint64_t));
    uint32_t* AV = vals ? (uint32_t*)malloc(nn * sizeof(uint32_t)) : NULL;
    uint32_t* BV = vals ? (uint32_t*)malloc(nn * sizeof(uint32_t)) : NULL;
    if (!A || !B || (vals && (!AV || !BV))) {
        free(A); free(B); free(AV); free(BV);
        return ORACLE_ENOMEM;
    }
    memcpy(A, keys, n * sizeof(uint64_t));
    if (vals) memcpy(AV, vals, n * sizeof(uint32_t));
    for (int p = 0; p < P; ++p) {
        int rc = oracle_counting_pass_u64(A, AV, B, BV, n, p * digit_bits, digit_bits);
        if (rc) { free(A); free(B); free(AV); free(BV); return rc; }
        uint64_t* t = A; A = B; B = t;
        uint32_t* tv = AV; AV = BV; BV = tv;
    }
    memcpy(out_keys, A, n * sizeof(uint64_t));
    if (vals && out_vals) memcpy(out_vals, AV, n * sizeof(uint32_t));
    free(A); free(B); free(AV); free(BV);
    return ORACLE_OK;
}

int oracle_radix_sort_u64(const uint64_t* keys, const uint32_t* vals, size_t n, int key_bits,
                          int digit_bits, uint64_t* out_keys, uint32_t* out_vals)
{
    return oracle_radix_sort_partial_u64(keys, vals, n, key_bits, digit_bits, -1, out_keys, out_vals);
}

/* ---------------------------------------------------------------------------
 * Sec. 2.2, Algorithm 1 (INSERTION-SORT), 0-based as printed: for j = 1 ..
 * len-1, take A[j] and shift every element that is strictly greater one slot
 * right, then drop the key into the gap.  The strict comparison keeps equal
 * keys in their order (stable).  The value moves with its key. */
static void insertion_sort(uint64_t* A, uint32_t* V, size_t len)
{
    for (size_t j = 1; j < len; ++j) {
        uint64_t key = A[j];
        uint32_t val = V ? V[j] : 0;
        size_t i = j; /* i is the paper's i + 1 so it stays unsigned */
        while (i > 0 && A[i - 1] > key) {
            A[i] = A[i - 1];
            if (V) V[i] = V[i - 1];
            --i;
        }
        A[i] = key;
        if (V) V[i] = val;
    }
}

/* Reading R3: the bucket of key k among nb buckets covering [min, max]. */
uint64_t oracle_bucket_index_u64(uint64_t key, uint64_t min_key, uint64_t max_key, uint64_t nb)
{
    u128 range = (u128)(max_key - min_key) + 1; /* up to 2^64 */
    u128 scaled = (u128)(key - min_key) * (u128)nb;
    return (uint64_t)(scaled / range);
}

/* Number of keys that fall into each of the nb buckets (the sizes of the lists
 * B[0..nb-1] after the insert loop of Algorithm 2). */
int oracle_bucket_counts_u64(const uint64_t* keys, size_t n, uint64_t min_key, uint64_t max_key,
                             uint64_t nb, uint64_t* counts)
{
    if (nb < 1 || min_key > max_key) return ORACLE_EARG;
    memset(counts, 0, sizeof(uint64_t) * nb);
    for (size_t i = 0; i < n; ++i) {
        if (keys[i] < min_key || keys[i] > max_key) return ORACLE_ERANGE;
        counts[oracle_bucket_index_u64(keys[i], min_key, max_key, nb)] += 1;
    }
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * Sec. 2.3, Algorithm 2 (BUCKET-SORT): insert every key, in input order, at
 * the tail of its bucket (readings R3, R4); sort each bucket with the
 * insertion sort of Algorithm 1; concatenate buckets 0 .. nb-1.  The buckets
 * are growable arrays instead of linked lists; the output is the same. */
int oracle_bucket_sort_u64(const uint64_t* keys, const uint32_t* vals, size_t n,
                           uint64_t min_key, uint64_t max_key, uint64_t nb,
                           uint64_t* out_keys, uint32_t* out_vals)
{
    if (nb < 1 || min_key > max_key) return ORACLE_EARG;
    for (size_t i = 0; i < n; ++i)
        if (keys[i] < min_key || keys[i] > max_key) return ORACLE_ERANGE;

    size_t* len = (size_t*)calloc(nb, sizeof(size_t));
    size_t* cap = (size_t*)calloc(nb, sizeof(size_t));
    uint64_t** BK = (uint64_t**)calloc(nb, sizeof(uint64_t*));
    uint32_t** BVv = (uint32_t**)calloc(nb, sizeof(uint32_t*));
    int rc = ORACLE_OK;
    if (!len || !cap || !BK || !BVv) { rc = ORACLE_ENOMEM; goto done; }

    /* insert A[i] into list B[bucket(A[i])] */
    for (size_t i = 0; i < n; ++i) {
        uint64_t b = oracle_bucket_index_u64(keys[i], min_key, max_key, nb);
        if (len[b] == cap[b]) {
            size_t nc = cap[b] ? 2 * cap[b] : 4;
            uint64_t* nk = (uint64_t*)realloc(BK[b], nc * sizeof(uint64_t));
            if (!nk) { rc = ORACLE_ENOMEM; goto done; }
            BK[b] = nk;
            if (vals) {
                uint32_t* nv = (uint32_t*)realloc(BVv[b], nc * sizeof(uint32_t));
                if (!nv) { rc = ORACLE_ENOMEM; goto done; }
                BVv[b] = nv;
            }
            cap[b] = nc;
        }
        BK[b][len[b]] = keys[i];
        if (vals) BVv[b][len[b]] = vals[i];
        len[b] += 1;
    }
    /* sort list B[i] with insertion sort, then concatenate */
    {
        size_t pos = 0;
        for (uint64_t b = 0; b < nb; ++b) {
            if (!len[b]) continue;
            insertion_sort(BK[b], vals ? BVv[b] : NULL, len[b]);
            memcpy(out_keys + pos, BK[b], len[b] * sizeof(uint64_t));
            if (vals && out_vals) memcpy(out_vals + pos, BVv[b], len[b] * sizeof(uint32_t));
            pos += len[b];
        }
    }
done:
    if (BK) for (uint64_t b = 0; b < nb; ++b) free(BK[b]);
    if (BVv) for (uint64_t b = 0; b < nb; ++b) free(BVv[b]);
    free(BK); free(BVv); free(len); free(cap);
    return rc;
}

/* Smallest and largest key: the bounds [min, max] that Algorithm 2 assumes
 * ("each integer is between 0 and M"), when the caller does not declare them. */
int oracle_minmax_u64(const uint64_t* keys, size_t n, uint64_t* min_key, uint64_t* max_key)
{
    if (n == 0) return ORACLE_EARG;
    uint64_t lo = keys[0], hi = keys[0];
    for (size_t i = 1; i < n; ++i) {
        if (keys[i] < lo) lo = keys[i];
        if (keys[i] > hi) hi = keys[i];
    }
    *min_key = lo;
    *max_key = hi;
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * Typed keys (beyond the paper, which sorts non-negative ints, Sec. 3.1).
 * The order of each key kind is written out as a comparison of the keys'
 * bits, width = 8 * key_bytes:
 *   kind 0, unsigned: the order of the unsigned integers;
 *   kind 1, signed (two's complement): a key with the sign bit set is below
 *           every key without it; keys of one sign compare as unsigned bits;
 *   kind 2, IEEE-754 binary float, totalOrder (IEEE 754-2008, 5.10): the bits
 *           are sign and magnitude; every key with the sign bit set is below
 *           every key without it; among non-negative keys the larger
 *           magnitude is larger, among negative keys the larger magnitude is
 *           smaller (so -0 < +0, and NaNs sit beyond the infinities, ordered
 *           by payload);
 *   descending: the reverse of that order.
 * The sort is a stable merge sort: equal keys keep their input order in both
 * directions.
 */
static int typed_less(uint64_t a, uint64_t b, int width, int kind)
{
    if (kind == 0)
        return a < b;
    const uint64_t sign = 1ull << (width - 1);
    const int sa = (a & sign) != 0, sb = (b & sign) != 0;
    if (sa != sb)
        return sa;  /* the negative one is smaller */
    if (kind == 1)
        return a < b;
    const uint64_t ma = a & ~sign, mb = b & ~sign;
    return sa ? (ma > mb) : (ma < mb);
}

static int typed_before(uint64_t a, uint64_t b, int width, int kind, int descending)
{
    return descending ? typed_less(b, a, width, kind) : typed_less(a, b, width, kind);
}

/* Merge sort of the index range [lo, hi) of idx by the keys; tmp is scratch.
 * The right element is taken only when it is strictly before the left one. */
static void merge_sort_idx(const uint64_t* keys, size_t* idx, size_t* tmp, size_t lo, size_t hi, int width,
                           int kind, int descending)
{
    if (hi - lo < 2)
        return;
    const size_t mid = lo + (hi - lo) / 2;
    merge_sort_idx(keys, idx, tmp, lo, mid, width, kind, descending);
    merge_sort_idx(keys, idx, tmp, mid, hi, width, kind, descending);
    size_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (typed_before(keys[idx[j]], keys[idx[i]], width, kind, descending))
            tmp[o++] = idx[j++];
        else
            tmp[o++] = idx[i++];
    }
    while (i < mid)
        tmp[o++] = idx[i++];
    while (j < hi)
        tmp[o++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (hi - lo) * sizeof(size_t));
}

int oracle_sort_typed_u64(const uint64_t* keys, const uint32_t* vals, size_t n, int key_bytes, int kind,
                          int descending, uint64_t* out, uint32_t* out_vals)
{
    if ((key_bytes != 4 && key_bytes != 8) || kind < 0 || kind > 2 || (n && (!keys || !out)))
        return ORACLE_EARG;
    if ((vals == NULL) != (out_vals == NULL))
        return ORACLE_EARG;
    const int width = 8 * key_bytes;
    if (width < 64) {
        for (size_t i = 0; i < n; ++i)
            if (keys[i] >> width)
                return ORACLE_EARG;
    }
    if (n == 0)
        return ORACLE_OK;
    size_t* idx = (size_t*)malloc(n * sizeof(size_t));
    size_t* tmp = (size_t*)malloc(n * sizeof(size_t));
    if (!idx || !tmp) {
        free(idx);
        free(tmp);
        return ORACLE_ENOMEM;
    }
    for (size_t i = 0; i < n; ++i)
        idx[i] = i;
    merge_sort_idx(keys, idx, tmp, 0, n, width, kind, descending);
    for (size_t i = 0; i < n; ++i) {
        out[i] = keys[idx[i]];
        if (vals)
            out_vals[i] = vals[idx[i]];
    }
    free(idx);
    free(tmp);
    return ORACLE_OK;
}
