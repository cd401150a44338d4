/*
 * rsort.h -- C ABI of a GB300 (sm_103a) integer-sort library implementing the
 * two methods compared in Horsmalahti, "Comparison of Bucket Sort and RADIX
 * Sort" (arXiv:1206.3511): LSD radix sort (Sec. 2.5, Algorithm 4, built from
 * the counting sort of Sec. 2.4, Algorithm 3) and bucket sort (Sec. 2.3,
 * Algorithm 2).
 *
 * The problem (Sec. 2): given a sequence of keys, produce a permutation of it
 * in nondecreasing order.  Both methods here are stable (the property is
 * defined in Sec. 2.1 and claimed for each method in Sec. 2.3 and 2.5): keys
 * that compare equal keep their input order, and an optional 32-bit value travels
 * with its key.  The output is therefore unique and every call is
 * bit-reproducible.
 *
 * Conventions shared by every call below:
 *   - All key, value, offset and workspace pointers are DEVICE pointers of the
 *     current CUDA device, except the h_* arrays of the host-buffer sorts
 *     (rs_sort_host_*, bs_sort_host_*, rs_sort_segmented_host_*).  The caller owns and allocates all of
 *     them; no sort call allocates device memory.
 *   - Calls are asynchronous: they validate their arguments on the host,
 *     enqueue kernels on `stream` and return.  Argument errors are returned
 *     synchronously and nothing is enqueued.  Errors found on the device (a
 *     key above 2^key_bits, a bounded wait that gave up) are recorded in a
 *     status word inside the workspace; read them with rs_get_status() before
 *     the next call on that workspace.
 *   - `stream` is a cudaStream_t (0 = the legacy default stream).
 *   - `ws` must be 256-byte aligned and at least rs_workspace_bytes(...)
 *     large.  A workspace may be reused by any number of calls issued on one
 *     stream; calls that use the same workspace concurrently on different
 *     streams race.
 *   - keys_in is read only.  keys_out == keys_in (in place) is allowed; any
 *     other overlap of inputs, outputs and workspace is an argument error
 *     where it can be detected and undefined otherwise.  The same holds for
 *     vals_in / vals_out.  vals_in and vals_out are both NULL (keys only) or
 *     both non-NULL.
 *   - Keys need only their natural alignment (4 bytes for u32, 8 for u64).
 *   - n = 0 is a no-op that returns RS_OK.
 *   - A single sort handles n <= RS_MAX_KEYS keys.
 */
#ifndef RSORT_H
#define RSORT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RS_API __attribute__((visibility("default")))
#else
#define RS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* rs_stream_t;

typedef enum rs_status {
    RS_OK = 0,
    RS_ERR_INVALID_ARG = 1,    /* bad pointer, size, alignment, overlap or parameter */
    RS_ERR_WORKSPACE = 2,      /* workspace NULL, misaligned or smaller than required */
    RS_ERR_KEY_RANGE = 3,      /* device: a key was >= 2^key_bits (or outside [min,max]) */
    RS_ERR_BUDGET = 4,         /* server: request can never fit the memory budget */
    RS_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    RS_ERR_DEVICE_TIMEOUT = 6, /* device: a bounded inter-block wait gave up */
    RS_ERR_NOT_READY = 7,      /* server: request still running */
    RS_ERR_SHUTDOWN = 8,       /* server: request cancelled by shutdown */
    RS_ERR_UNSUPPORTED = 9,    /* configuration not compiled into this build */
    RS_ERR_CHECK_FAILED = 10   /* device, checked mode (RS_CHECKED=1): an output was not in order */
} rs_status;

/* Largest n for one (unsegmented) sort: per-block digit counts travel in the
 * 30-bit count field of the inter-block status words. */
#define RS_MAX_KEYS ((size_t)1 << 30)

/* Algorithms for rs_workspace_bytes(). */
#define RS_ALGO_RADIX 0
#define RS_ALGO_BUCKET 1

/* Kernel shape of one radix sort.  digit_bits is the D of a D-bit digit
 * (Sec. 2.5 leaves the digit base open); a sort makes ceil(key_bits / D)
 * passes.  Every valid configuration gives bit-identical output. */
typedef struct rs_config {
    int digit_bits;       /* 4 .. 11 */
    int block_threads;    /* threads per block of the scatter pass */
    int items_per_thread; /* keys per thread of the scatter pass */
} rs_config;

/* Human-readable name of a status code (static string, never NULL). */
RS_API const char* rs_status_string(rs_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
RS_API int rs_version(void);

/* Default kernel shape for keys of `key_bytes` (4 or 8) bytes, with or
 * without values, for n keys.  Returns RS_ERR_INVALID_ARG on bad sizes. */
RS_API rs_status rs_default_config(int key_bytes, int has_values, size_t n, rs_config* out);

/* Number of configurations compiled for (key_bytes, has_values) and the i-th
 * of them (i = 0 .. count-1); these are the candidates an autotuner may try. */
RS_API int rs_config_count(int key_bytes, int has_values);
RS_API rs_status rs_config_get(int key_bytes, int has_values, int i, rs_config* out);

/* Workspace bytes for one call of the given algorithm, valid for every
 * compiled configuration with digit_bits <= 8.  key_bytes: 4 or 8.  key_bits: 0 means the full key
 * width.  num_buckets: bucket count for RS_ALGO_BUCKET (0 = max(1, n/16));
 * ignored for radix.  in_place: nonzero if keys_out will equal keys_in (the
 * workspace is the same either way).
 * Returns 0 for invalid arguments. */
RS_API size_t rs_workspace_bytes(int algo, int key_bytes, int has_values, size_t n, int key_bits,
                          size_t num_buckets, int in_place);

/* Workspace bytes of a radix sort run with one explicit kernel shape (needed
 * for shapes with digit_bits > 8, which rs_workspace_bytes does not cover).
 * Returns 0 for invalid arguments or a shape that is not compiled. */
RS_API size_t rs_workspace_bytes_cfg(int key_bytes, int has_values, size_t n, int key_bits, const rs_config* cfg);

/* ---------------------------------------------------------------------------
 * LSD radix sort, Sec. 2.5 Algorithm 4: d = ceil(key_bits / D) stable passes,
 * least significant digit first, each pass a counting sort (Sec. 2.4,
 * Algorithm 3) on one D-bit digit.  Every key must be < 2^key_bits
 * (key_bits 1..32 for u32, 1..64 for u64; 0 means the full width); a larger
 * key is reported as RS_ERR_KEY_RANGE by rs_get_status() and leaves the output
 * unspecified (but every write stays inside keys_out / vals_out).
 * Result: keys_out[0..n) nondecreasing; vals_out[i] is the value that came
 * with keys_out[i]; equal keys in input order.
 */
RS_API rs_status rs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                      uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                      rs_stream_t stream);
RS_API rs_status rs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                      uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                      rs_stream_t stream);

/* Same as rs_sort_u32/u64 with an explicit kernel shape (NULL = default).
 * RS_ERR_UNSUPPORTED if that shape is not compiled. */
RS_API rs_status rs_sort_u32_ex(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                         uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                         rs_stream_t stream, const rs_config* cfg);
RS_API rs_status rs_sort_u64_ex(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                         uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                         rs_stream_t stream, const rs_config* cfg);

/* Typed keys: the radix sort of rs_sort_u32/u64 over another order.  The
 * paper sorts non-negative `int` keys (Sec. 3.1); this call extends it to
 * signed integers, IEEE-754 floats and descending order by sorting the keys'
 * order-preserving unsigned images: a signed key flips its sign bit; a float
 * flips its sign bit when non-negative and all bits when negative, so floats
 * follow the standard's totalOrder (-NaN < -inf < ... < -0 < +0 < ... < +inf
 * < +NaN, NaNs by payload); descending complements the image.  The images
 * are formed as the keys are loaded and undone as they are stored: the output
 * holds the original key bits.  Stable in every mode (equal keys keep input
 * order, also when descending).
 * key_kind: RS_KEY_UINT, RS_KEY_INT or RS_KEY_FLOAT; key_bytes 4 or 8;
 * every bit is significant (no key_bits).  Workspace: rs_workspace_bytes(
 * RS_ALGO_RADIX, key_bytes, has_values, n, 0, 0, in_place).  Layout, aliasing
 * and errors as rs_sort_u32/u64. */
#define RS_KEY_UINT 0
#define RS_KEY_INT 1
#define RS_KEY_FLOAT 2
RS_API rs_status rs_sort_typed(int key_kind, int key_bytes, int descending, const void* keys_in, void* keys_out,
                               const uint32_t* vals_in, uint32_t* vals_out, size_t n, void* ws, size_t ws_bytes,
                               rs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Bucket sort, Sec. 2.3 Algorithm 2: every key goes to bucket
 *     b(k) = floor((k - min_key) * num_buckets / (max_key - min_key + 1))
 * (exact; the paper's n * A[i] / M with an inclusive key range), in input
 * order; every bucket is sorted (buckets of up to 48 keys by a stable rank
 * sort that makes insertion sort's comparisons, Sec. 2.2 Algorithm 1, for all
 * keys at once; larger ones by a stable radix sort of the bucket's key
 * range); the buckets are concatenated in bucket order.  The result is the
 * stable sort of the keys, identical to rs_sort_*.
 * min_key > max_key: the bounds are the keys' own minimum and maximum,
 * computed on the device.  Otherwise every key must lie in [min_key,
 * max_key]; a key outside is reported as RS_ERR_KEY_RANGE by rs_get_status()
 * (output unspecified, writes stay inside the outputs).
 * num_buckets: 0 means max(1, n/16); at most 2^32.
 * Workspace: rs_workspace_bytes(RS_ALGO_BUCKET, key_bytes, has_values, n, 0,
 * num_buckets, in_place).  In place (keys_out == keys_in) is allowed.
 */
RS_API rs_status bs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                             uint32_t* vals_out, size_t n, uint32_t min_key, uint32_t max_key, size_t num_buckets,
                             void* ws, size_t ws_bytes, rs_stream_t stream);
RS_API rs_status bs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                             uint32_t* vals_out, size_t n, uint64_t min_key, uint64_t max_key, size_t num_buckets,
                             void* ws, size_t ws_bytes, rs_stream_t stream);

/* The bucket counts of Algorithm 2's insert step: d_counts[b] = the number of
 * keys with b(k) = b (the formula above), for b in [0, num_buckets).
 * d_counts: DEVICE array of num_buckets uint32, overwritten.  Requires
 * min_key <= max_key and 1 <= num_buckets <= 2^32; a key outside [min_key,
 * max_key] is not counted and is reported as RS_ERR_KEY_RANGE by
 * rs_get_status().  Workspace: at least 1024 bytes (any bucket-sort
 * workspace will do).  One global atomic per key: a building block and a
 * check of the bucket function, not a fast path. */
RS_API rs_status bs_bucket_counts_u32(const uint32_t* keys, size_t n, uint32_t min_key, uint32_t max_key,
                                      size_t num_buckets, uint32_t* d_counts, void* ws, size_t ws_bytes,
                                      rs_stream_t stream);
RS_API rs_status bs_bucket_counts_u64(const uint64_t* keys, size_t n, uint64_t min_key, uint64_t max_key,
                                      size_t num_buckets, uint32_t* d_counts, void* ws, size_t ws_bytes,
                                      rs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Building blocks: one step of the radix path each.
 *
 * rs_digit_counts_*: the counting loop of Algorithm 3 for every pass of
 * Algorithm 4 in one read of the keys.  counts_out (device, uint32,
 * ceil(key_bits/D) * 2^D entries, row p = pass p) receives
 * counts_out[p * 2^D + d] = #{i : (keys[i] >> (p*D)) & (2^D-1) == d}.
 * digit_bits 4..11.
 */
RS_API rs_status rs_digit_counts_u32(const uint32_t* keys, size_t n, int key_bits, int digit_bits,
                              uint32_t* counts_out, void* ws, size_t ws_bytes, rs_stream_t stream);
RS_API rs_status rs_digit_counts_u64(const uint64_t* keys, size_t n, int key_bits, int digit_bits,
                              uint32_t* counts_out, void* ws, size_t ws_bytes, rs_stream_t stream);

/* rs_counting_pass_*: one stable counting sort (Algorithm 3) of the whole
 * array on the digit (key >> shift) & (2^digit_bits - 1), digit_bits 4..11,
 * shift 0..(key width - 1).  keys_out must not overlap keys_in (likewise the
 * values).  Workspace: rs_workspace_bytes(RS_ALGO_RADIX, ...) for the same n. */
RS_API rs_status rs_counting_pass_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                               uint32_t* vals_out, size_t n, int shift, int digit_bits, void* ws,
                               size_t ws_bytes, rs_stream_t stream);
RS_API rs_status rs_counting_pass_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                               uint32_t* vals_out, size_t n, int shift, int digit_bits, void* ws,
                               size_t ws_bytes, rs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Segmented sort: many independent arrays in one call.  Segment s is
 * [d_seg_offsets[s], d_seg_offsets[s+1]) of the key (and value) arrays; each
 * segment is sorted as rs_sort_u32/u64 would sort it alone (Algorithm 4 per
 * segment, stable).  d_seg_offsets: DEVICE array of nseg+1 nondecreasing
 * uint64 offsets with d_seg_offsets[nseg] = n_total <= the length of the
 * arrays; a segment may be empty; one segment may hold at most
 * RS_MAX_KEYS - 1 keys.  Segments of up to 4096 keys are sorted inside one
 * thread block in shared memory, larger ones by segmented scatter passes; the
 * classification is done on the device, so the call never waits for the GPU.
 * An offsets table that decreases, runs past n_total or has a segment above
 * the limit is reported as RS_ERR_INVALID_ARG by rs_get_status(): such
 * segments are dropped (their output is unspecified), every other segment is
 * sorted, and nothing is written outside [0, n_total) of the arrays or the
 * workspace.  A key with bits at or above key_bits is reported as
 * RS_ERR_KEY_RANGE (that segment's output is unspecified).
 * Workspace: rs_segmented_workspace_bytes(key_bytes, has_values, n_total,
 * nseg, key_bits).  In place (keys_out == keys_in) is allowed.
 */
RS_API size_t rs_segmented_workspace_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg,
                                           int key_bits);
RS_API rs_status rs_sort_segmented_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                       uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                       size_t n_total, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream);
RS_API rs_status rs_sort_segmented_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                       uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                       size_t n_total, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream);
/* Segmented bucket sort: each segment [d_seg_offsets[s], d_seg_offsets[s+1])
 * of the arrays is bucket-sorted on its own, as bs_sort_u32/u64 would sort it
 * alone (Sec. 2.3, Algorithm 2, per segment; stable).  Segment s of n_s keys
 * gets max(1, floor(n_s / keys_per_bucket)) buckets (keys_per_bucket 0 =
 * 16, the n/16 rule of bs_sort_*; 1 gives the paper's n buckets) over the
 * range [min_key, max_key] when min_key <= max_key (every key of every
 * segment must lie in it; a key outside is reported as RS_ERR_KEY_RANGE), or
 * over that segment's own smallest and largest key when min_key > max_key
 * (found on the device).  Segments of up to 4096 keys are bucket-sorted whole
 * inside one thread block; larger ones are partitioned by their bucket ids in
 * two segmented one-sweep levels, every partition of up to 4096 keys is then
 * sorted bucket by bucket in shared memory, and a partition still larger when
 * the bucket bits run out (skewed keys) is radix-sorted on the key bits its
 * buckets span.  Offsets follow rs_sort_segmented_u32's rules (DEVICE array
 * of nseg+1 offsets, d_seg_offsets[nseg] <= n_total, errors reported on the
 * device as RS_ERR_INVALID_ARG, no write outside the arrays).  The
 * classification is done on the device: the call never waits for the GPU.
 * Workspace: bs_segmented_workspace_bytes(key_bytes, has_values, n_total,
 * nseg, keys_per_bucket), valid for any bounds.  In place is allowed.
 * RS_ERR_INVALID_ARG (synchronous): mismatched value pointers, misaligned or
 * overlapping arrays, keys_per_bucket > 2^30, a u32 max_key above 2^32 - 1.
 */
RS_API size_t bs_segmented_workspace_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg,
                                           size_t keys_per_bucket);
RS_API rs_status bs_sort_segmented_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                       uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                       size_t n_total, uint32_t min_key, uint32_t max_key, size_t keys_per_bucket,
                                       void* ws, size_t ws_bytes, rs_stream_t stream);
RS_API rs_status bs_sort_segmented_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                       uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                       size_t n_total, uint64_t min_key, uint64_t max_key, size_t keys_per_bucket,
                                       void* ws, size_t ws_bytes, rs_stream_t stream);
/* Same with an explicit kernel shape for the scatter passes of the large
 * segments (NULL = default).  Every shape rs_config_get lists is compiled for
 * segmented passes at digit_bits = 8; another digit width or shape gives
 * RS_ERR_UNSUPPORTED.  The output does not depend on the shape. */
RS_API rs_status rs_sort_segmented_u32_ex(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                          uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                          size_t n_total, int key_bits, void* ws, size_t ws_bytes,
                                          rs_stream_t stream, const rs_config* cfg);
RS_API rs_status rs_sort_segmented_u64_ex(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                          uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg,
                                          size_t n_total, int key_bits, void* ws, size_t ws_bytes,
                                          rs_stream_t stream, const rs_config* cfg);

/* ---------------------------------------------------------------------------
 * Plans: one sort call with fixed buffers and sizes, captured once into a
 * CUDA graph and replayed by rs_plan_launch with a single host launch (the
 * segmented sort of many arrays then costs one launch per call).  The
 * planned call is rs_sort_* (RS_PLAN_RADIX), bs_sort_* (RS_PLAN_BUCKET) or
 * rs_sort_segmented_* (RS_PLAN_SEGMENTED, n = n_total) with the arguments in
 * the descriptor; argument errors are returned by rs_plan_create.
 * autotune (radix and segmented): every compiled kernel shape (radix: whose
 * workspace fits ws_bytes; segmented: every 8-bit shape) is timed on the
 * plan's buffers and the fastest is kept (all shapes give identical bits);
 * results are cached per GPU, algorithm, key width, values, key_bits and
 * floor(log2 n) for the life of the process.
 * rs_plan_create runs the planned sort at least once (more when tuning) on
 * the plan's buffers and waits for it.  The buffers must stay valid for the
 * life of the plan; a plan must not be launched concurrently with itself.
 */
#define RS_PLAN_RADIX 0
#define RS_PLAN_BUCKET 1
#define RS_PLAN_SEGMENTED 2
typedef struct rs_plan rs_plan;
typedef struct rs_plan_desc {
    int algo;
    int key_bytes;
    const void* keys_in;
    void* keys_out;
    const uint32_t* vals_in;
    uint32_t* vals_out;
    size_t n;
    int key_bits;
    uint64_t min_key, max_key; /* bucket */
    size_t num_buckets;        /* bucket */
    const uint64_t* d_seg_offsets; /* segmented */
    size_t nseg;                   /* segmented */
    void* ws;
    size_t ws_bytes;
    int autotune;
} rs_plan_desc;
RS_API rs_status rs_plan_create(const rs_plan_desc* desc, rs_plan** out);
RS_API rs_status rs_plan_launch(rs_plan* plan, rs_stream_t stream);
/* The kernel shape in use (radix and segmented plans; zeros otherwise), the number of
 * kernel nodes in the graph, and the tuned time per sort in ms (-1 if not
 * tuned in this call). */
RS_API rs_status rs_plan_info(const rs_plan* plan, rs_config* cfg, size_t* kernel_nodes, float* tuned_ms);
RS_API void rs_plan_destroy(rs_plan* plan);

/* Autotuning results, kept across processes (no counterpart in the paper:
 * the digit base of Sec. 2.5 is left open, and the autotuner picks it per
 * GPU).  A plan's autotuner caches the shape it picks per (GPU name,
 * algorithm, key width, values, key_bits, floor(log2 n)).  The cache can be
 * written to and merged from a file of one JSON object per line, e.g.
 *   {"gpu": "NVIDIA GB300", "algo": 0, "key_bytes": 4, "values": 0,
 *    "key_bits": 32, "log2n": 26, "digit_bits": 8, "block_threads": 256,
 *    "items_per_thread": 22}
 * Lines that do not parse, or name a shape this build does not compile, are
 * skipped.  With the environment variable RS_TUNE_CACHE set to a path, plans
 * merge that file before their first tuning and rewrite it (through a
 * temporary file and a rename) after each new result.
 *   rs_tune_cache_load: entries merged from path, or -1 if it cannot be read.
 *   rs_tune_cache_save: entries written to path, or -1 on an I/O error.
 *   rs_tune_cache_size: entries in the process's cache.
 *   rs_tune_cache_clear: forget every entry (files are not touched).
 * Thread-safe; no GPU needed.
 *
 * Other environment switches (read once per process): RS_DIGIT_BITS (4..11)
 * sets the digit width of radix sorts that name no kernel shape (default 8);
 * RS_SPIN_LIMIT sets the poll limit of the bounded inter-block waits unless
 * rs_set_debug has set one; RS_CHECKED=1 makes rs_sort_*, rs_sort_typed and
 * bs_sort_* verify on the device that their output is in order, recording
 * RS_ERR_CHECK_FAILED in the status word if it is not. */
RS_API int rs_tune_cache_load(const char* path);
RS_API int rs_tune_cache_save(const char* path);
RS_API int rs_tune_cache_size(void);
RS_API void rs_tune_cache_clear(void);

/* ---------------------------------------------------------------------------
 * Sort server (continuous batching).  Requests arrive at any time from any
 * host thread; a dispatcher thread admits them, oldest first, while the
 * memory they need fits under budget_bytes, and keeps up to num_streams
 * launches in flight on separate streams so their work overlaps on the GPU.
 * Waiting requests of at most batch_max_keys keys are packed, up to
 * max_batch at a time, into one segmented sort (their keys are gathered into
 * the pool, sorted per segment and copied back): radix requests with the same
 * key type, value presence and key_bits through rs_sort_segmented_*, bucket
 * requests with the same key type and value presence, the default bucket
 * count (num_buckets 0 or max(1, n/16)) and the same declared bounds (or
 * bounds computed for each) through bs_sort_segmented_*; other requests run
 * as single sorts.  A bucket request of 4-byte keys with max_key above
 * 2^32 - 1 (and min_key <= max_key) is refused with RS_ERR_INVALID_ARG.  Each
 * request's output is exactly what rs_sort_* / bs_sort_* would produce for
 * it alone.
 *
 * pool/pool_bytes: caller-owned DEVICE memory (256-byte aligned) from which
 * the server takes workspaces and batch staging; the server never allocates
 * device memory.  budget_bytes (0 = pool_bytes): admission budget over every
 * admitted request's own inputs and outputs, its workspace and any staging.
 * A request that can never fit is refused at submit with RS_ERR_BUDGET.
 * Request buffers must stay valid and untouched until the request is done.
 * The server uses the CUDA device that is current at rs_server_create.
 */
typedef struct rs_server rs_server;
typedef struct rs_server_config {
    void* pool;
    size_t pool_bytes;
    size_t budget_bytes;
    int num_streams;        /* 1 .. 64 */
    int max_batch;          /* requests per batched launch, >= 1 (1 = no batching) */
    size_t batch_max_keys;  /* largest request that may be batched (0 = 262144) */
} rs_server_config;
typedef struct rs_request {
    int algo;       /* RS_ALGO_RADIX or RS_ALGO_BUCKET */
    int key_bytes;  /* 4 or 8 */
    const void* keys_in;
    void* keys_out;
    const uint32_t* vals_in; /* NULL for keys only */
    uint32_t* vals_out;
    size_t n;
    int key_bits;           /* radix: as rs_sort_*; ignored for bucket */
    uint64_t min_key, max_key; /* bucket: as bs_sort_* (min > max: computed) */
    size_t num_buckets;     /* bucket: as bs_sort_* */
} rs_request;
typedef struct rs_result {
    rs_status status;   /* RS_ERR_NOT_READY while queued or running */
    double t_arrive_ms; /* host steady-clock times: submit, launch, completion seen */
    double t_start_ms;
    double t_done_ms;
} rs_result;
typedef struct rs_server_stats {
    uint64_t submitted, completed, rejected, queued;
    size_t in_use_bytes, max_in_use_bytes, budget_bytes;
    uint64_t batches, batched_requests;
    uint64_t max_queued; /* the longest the queue of waiting requests has been */
} rs_server_stats;

RS_API rs_status rs_server_create(const rs_server_config* cfg, rs_server** out);
/* Queue a request; *ticket identifies it.  RS_ERR_BUDGET: it can never fit;
 * RS_ERR_SHUTDOWN: the server is being destroyed. */
RS_API rs_status rs_server_submit(rs_server* s, const rs_request* req, uint64_t* ticket);
/* Status of a request without waiting (RS_ERR_NOT_READY while not done). */
RS_API rs_status rs_server_poll(rs_server* s, uint64_t ticket, rs_result* out);
/* Wait up to timeout_ms (< 0: forever) for a request; its status, or
 * RS_ERR_NOT_READY on timeout.  A finished request's status is the host-side
 * result of launching it (argument or CUDA errors) or, when that succeeded,
 * the device status word of its sort as rs_get_status() would read it
 * (RS_ERR_KEY_RANGE for a key above key_bits or outside the declared bucket
 * range, RS_ERR_DEVICE_TIMEOUT, ...).  A batched request shares the status
 * word of its batch: a device error in one request of a batch is reported by
 * every request of that batch. */
RS_API rs_status rs_server_wait(rs_server* s, uint64_t ticket, int timeout_ms);
/* Forget a finished request: its record (status and times) is freed and the
 * ticket becomes unknown (later calls on it return RS_ERR_INVALID_ARG).  A
 * server keeps every record until it is released or destroyed.
 * RS_ERR_NOT_READY if the request is still queued or running. */
RS_API rs_status rs_server_release(rs_server* s, uint64_t ticket);
RS_API rs_status rs_server_get_stats(rs_server* s, rs_server_stats* out);
/* Stop accepting requests; finish (cancel_pending = 0) or cancel (nonzero:
 * queued requests end with RS_ERR_SHUTDOWN) the queue, wait for launches in
 * flight, release streams and the dispatcher.  The pool is not freed. */
RS_API rs_status rs_server_destroy(rs_server* s, int cancel_pending);

/* ---------------------------------------------------------------------------
 * Sorting without a caller-provided workspace.  The paper has no counterpart:
 * this exists for callers that cannot allocate device memory (code running
 * where cudaMalloc is not allowed or not available, or that cannot own an
 * extra buffer).
 *
 * rs_sort_u32_noalloc: same result as rs_sort_u32 (stable LSD radix sort of
 * uint32 keys, optional uint32 values, key_bits 0..32), but its scratch is a
 * fixed 9 MiB array inside the library's device memory, so the call allocates
 * nothing.  Every GPU that loads the library holds that array until the
 * process exits.  n must be <= RS_NOALLOC_MAX_KEYS, otherwise
 * RS_ERR_INVALID_ARG is returned and nothing is enqueued.  All calls share
 * the one array: calls that overlap on the GPU (other streams, or unordered
 * host threads) race and give wrong results.  The first call on each device
 * looks up the array's device address; make it before any stream capture on
 * that device.  Device-side errors of these calls (a key above 2^key_bits, a
 * bounded wait that gave up) are recorded in the shared array and are not
 * readable through this API; use rs_sort_u32 with a workspace when they
 * matter.  Argument rules otherwise as rs_sort_u32.
 */
#define RS_NOALLOC_MAX_KEYS ((size_t)1 << 20)
RS_API rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                     uint32_t* vals_out, size_t n, int key_bits, rs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Sorting arrays that live in host memory.  The paper has no counterpart (its
 * arrays are in the one memory of a CPU); these calls solve Sec. 2's problem
 * for a caller whose keys are in host memory.
 *
 * rs_sort_host_u32 / rs_sort_host_u64 (radix) and bs_sort_host_u32 /
 * bs_sort_host_u64 (bucket) enqueue on `stream`, in this order: a copy of the
 * keys (and values) from host memory into `dev_buf`; the same sort as
 * rs_sort_u32 / rs_sort_u64 or bs_sort_u32 / bs_sort_u64, run in place
 * there; and a copy of the sorted keys (and values) back into host memory.
 * The result in h_keys_out / h_vals_out equals that of the device call.
 *   - h_keys_in, h_keys_out, h_vals_in, h_vals_out are HOST pointers with the
 *     keys' natural alignment (device memory is RS_ERR_INVALID_ARG).
 *     h_keys_out == h_keys_in is allowed, likewise for the values; any other
 *     overlap is RS_ERR_INVALID_ARG.  The values are both NULL (keys only)
 *     or both non-NULL.
 *   - With page-locked host memory (cudaHostAlloc, cudaHostRegister) the call
 *     returns at once and the copies run asynchronously; the host buffers
 *     must then stay untouched until the stream has passed the call.  With
 *     pageable memory the CUDA runtime stages the copies and the call may
 *     block the calling thread.
 *   - dev_buf is a DEVICE buffer owned by the caller, 256-byte aligned and at
 *     least rs_host_sort_bytes(algo, key_bytes, has_values, n, key_bits,
 *     num_buckets) bytes (RS_ERR_WORKSPACE otherwise).  It holds the sort's
 *     workspace at its start, so rs_get_status(dev_buf, stream) reads the
 *     device status of the call, then the keys and the values.  Calls on
 *     different streams with different dev_buf run concurrently: one call's
 *     copies overlap another call's sort.
 *   - key_bits (radix), min_key, max_key and num_buckets (bucket) as for the
 *     device calls.
 * rs_host_sort_bytes returns 0 for an invalid algo, key_bytes, key_bits, n or
 * num_buckets.
 */
RS_API size_t rs_host_sort_bytes(int algo, int key_bytes, int has_values, size_t n, int key_bits,
                                 size_t num_buckets);
RS_API rs_status rs_sort_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out, const uint32_t* h_vals_in,
                                  uint32_t* h_vals_out, size_t n, int key_bits, void* dev_buf,
                                  size_t dev_buf_bytes, rs_stream_t stream);
RS_API rs_status rs_sort_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out, const uint32_t* h_vals_in,
                                  uint32_t* h_vals_out, size_t n, int key_bits, void* dev_buf,
                                  size_t dev_buf_bytes, rs_stream_t stream);
RS_API rs_status bs_sort_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out, const uint32_t* h_vals_in,
                                  uint32_t* h_vals_out, size_t n, uint32_t min_key, uint32_t max_key,
                                  size_t num_buckets, void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream);
RS_API rs_status bs_sort_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out, const uint32_t* h_vals_in,
                                  uint32_t* h_vals_out, size_t n, uint64_t min_key, uint64_t max_key,
                                  size_t num_buckets, void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream);

/* The segmented sort of rs_sort_segmented_u32_ex / _u64_ex on host arrays:
 * h_seg_offsets is a HOST array of nseg+1 uint64 offsets (same rules as
 * d_seg_offsets), copied into dev_buf with the keys and values; cfg as for
 * the _ex calls (NULL = default).  dev_buf: at least
 * rs_segmented_host_bytes(key_bytes, has_values, n_total, nseg, key_bits)
 * bytes.  Other rules as for rs_sort_host_u32 above; the offsets must not
 * overlap the outputs.  nseg = 0 or n_total = 0 is a no-op. */
RS_API size_t rs_segmented_host_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg, int key_bits);
RS_API rs_status rs_sort_segmented_host_u32(const uint32_t* h_keys_in, uint32_t* h_keys_out,
                                            const uint32_t* h_vals_in, uint32_t* h_vals_out,
                                            const uint64_t* h_seg_offsets, size_t nseg, size_t n_total,
                                            int key_bits, void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream,
                                            const rs_config* cfg);
RS_API rs_status rs_sort_segmented_host_u64(const uint64_t* h_keys_in, uint64_t* h_keys_out,
                                            const uint32_t* h_vals_in, uint32_t* h_vals_out,
                                            const uint64_t* h_seg_offsets, size_t nseg, size_t n_total,
                                            int key_bits, void* dev_buf, size_t dev_buf_bytes, rs_stream_t stream,
                                            const rs_config* cfg);

/* ---------------------------------------------------------------------------
 * Device status.
 *
 * rs_get_status: waits for `stream`, then reads and clears the status word
 * kept in the workspace header.  Every call that takes a workspace clears
 * that word when it starts on the device, so the word describes the most
 * recent such call: RS_OK, or the first device error it recorded
 * (RS_ERR_KEY_RANGE, RS_ERR_DEVICE_TIMEOUT).  Returns RS_ERR_CUDA if the
 * stream itself failed.  ws must have been passed to at least one call.
 */
RS_API rs_status rs_get_status(const void* ws, rs_stream_t stream);

/* Test hooks for the bounded inter-block waits.  spin_limit: polls before a
 * wait gives up (0 = library default, about a second of polling).
 * stall_tile: if >= 0, the block that handles that tile of every scatter pass
 * never publishes its counts, so later blocks wait until spin_limit runs out
 * and report RS_ERR_DEVICE_TIMEOUT (the output is then unspecified, but all
 * writes stay inside the output arrays).  Process-wide; not thread safe;
 * reset with rs_set_debug(0, -1). */
RS_API void rs_set_debug(uint32_t spin_limit, int stall_tile);

/* ---------------------------------------------------------------------------
 * Kernel timing and launch counting (instrumentation for benchmarks; the
 * paper measured whole sorts with clock(), Sec. 3.1).
 *
 * rs_profile_enable(1): from now on the library records a CUDA event before
 * and after every kernel it launches, on the stream of that launch.
 * rs_profile_read: waits for the recorded events, adds their durations per
 * kernel kind into out[0 .. cap), returns the number of kinds filled (or -1
 * on a CUDA error) and forgets the records.  rs_launch_count: number of
 * kernels this library has launched since it was loaded (always counted).
 */
typedef struct rs_kernel_stat {
    char name[32];
    uint64_t launches;
    double total_ms;
} rs_kernel_stat;
RS_API void rs_profile_enable(int enable);
RS_API int rs_profile_read(rs_kernel_stat* out, int cap);
RS_API uint64_t rs_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RSORT_H */
