// rs_segmented.h -- internal interface of the segmented-sort host code,
// shared with the bucket sort.
#pragma once

#include <algorithm>

#include "rs_radix.h"
#include "rs_segmented.cuh"

namespace rs {

// Digit width of the segmented scatter passes.
constexpr int kSegDigitBits = 8;

// Shared-memory sort capacity: segments of at most this many keys are
// sorted inside one block.
constexpr int kLocalBlock = 256;
constexpr int kLocalItems = 16;
constexpr uint32_t kLocalCap = kLocalBlock * kLocalItems;

#ifndef RS_BUCKET_BLOCK  // u32 keys-only bucket partition passes: 256 x 28, 3 blocks/SM
#define RS_BUCKET_BLOCK 256
#define RS_BUCKET_ITEMS 28
#define RS_BUCKET_MINB 3
#endif

// Kernel shapes of the segmented and bucket scatter passes.
template <typename KeyT, bool VALS>
struct SegShape;
template <>
struct SegShape<uint32_t, false> {
    static constexpr int kBlock = 256, kItems = 22, kMinB = 4, kTile = kBlock * kItems;
};
template <>
struct SegShape<uint32_t, true> {
    static constexpr int kBlock = 256, kItems = 12, kMinB = 4, kTile = kBlock * kItems;
};
template <>
struct SegShape<uint64_t, false> {
    static constexpr int kBlock = 256, kItems = 12, kMinB = 4, kTile = kBlock * kItems;
};
template <>
struct SegShape<uint64_t, true> {
    static constexpr int kBlock = 256, kItems = 10, kMinB = 3, kTile = kBlock * kItems;
};

// Kernel shapes of the bucket sort's partition passes.  Their digit carries
// the bucket parameters (and computes the bucket id of every key twice),
// which takes registers the radix passes spend on keys, so they have their
// own shape.  Measured at 100M uniform u32 keys (whole bucket sort): 256 x 28
// 2.74 ms, 256 x 32 2.75, 384 x 18 2.81, 384 x 12 2.93 (the only one of them
// without a spill); larger tiles win as in the radix passes.
template <typename KeyT, bool VALS>
struct BucketShape : SegShape<KeyT, VALS> {};
template <>
struct BucketShape<uint32_t, false> {
    static constexpr int kBlock = RS_BUCKET_BLOCK, kItems = RS_BUCKET_ITEMS, kMinB = RS_BUCKET_MINB,
                         kTile = kBlock * kItems;
};

// Keys per tile of the bucket passes, and the smallest tile of the bucket
// and segmented radix passes (workspace sizing of the bucket sorts).
inline uint32_t bucket_tile_keys(int key_bytes, bool vals) {
    if (key_bytes == 4) return vals ? BucketShape<uint32_t, true>::kTile : BucketShape<uint32_t, false>::kTile;
    return vals ? BucketShape<uint64_t, true>::kTile : BucketShape<uint64_t, false>::kTile;
}

// One segmented scatter pass with an explicit kernel shape.
template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB, typename DigitOp>
cudaError_t launch_seg_pass_shape(const SegPassParams<DigitOp>& sp, size_t grid, cudaStream_t s) {
    using Shape = OnesweepShape<KeyT, VALS, BLOCK, ITEMS>;
    auto kern = k_onesweep_seg<KeyT, VALS, BLOCK, ITEMS, MINB, DigitOp>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    const size_t most = DigitOp::kStageDigit ? pass_smem_bytes<Shape, DigitOp>(8) : max_fitting_pass_smem<Shape>();
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t smem = pass_smem_bytes<Shape, DigitOp>(sp.base.digit_bits);
    if (smem > most) return cudaErrorInvalidValue;
    grid = std::min<size_t>(grid, (size_t)resident_grid(kern, BLOCK, smem));
    KernelScope scope("onesweep_seg_pass", s);
    kern<<<(unsigned)(grid ? grid : 1), BLOCK, smem, s>>>(sp);
    return cudaGetLastError();
}

// One segmented scatter pass with the default shape of its key type (the
// bucket shape for bucket-id digits).
template <typename KeyT, bool VALS, typename DigitOp>
cudaError_t launch_seg_pass(const SegPassParams<DigitOp>& sp, size_t grid, cudaStream_t s) {
    using S = SegShape<KeyT, VALS>;
    return launch_seg_pass_shape<KeyT, VALS, S::kBlock, S::kItems, S::kMinB, DigitOp>(sp, grid, s);
}
template <typename KeyT, bool VALS, typename DigitOp>
cudaError_t launch_bucket_seg_pass(const SegPassParams<DigitOp>& sp, size_t grid, cudaStream_t s) {
    using S = BucketShape<KeyT, VALS>;
    return launch_seg_pass_shape<KeyT, VALS, S::kBlock, S::kItems, S::kMinB, DigitOp>(sp, grid, s);
}

// Kernel shapes compiled for the segmented radix passes (8-bit digits): the
// same shapes as the plain radix sort; index 0 of each key type is SegShape.
int seg_shape_count(int key_bytes, bool vals);
// Index of the shape (block, items), or -1 if it is not compiled.
int seg_shape_find(int key_bytes, bool vals, int block, int items);
// Block size and keys per thread of shape i; false if there is none.
bool seg_shape_get(int key_bytes, bool vals, int i, int* block, int* items);
// Keys per tile of shape i, and the smallest over all shapes (workspace sizing).
uint32_t seg_shape_tile(int key_bytes, bool vals, int i);
uint32_t seg_min_tile(int key_bytes, bool vals);

template <typename KeyT, typename Digits>
cudaError_t launch_seg_counts(const KeyT* keys, const SegDesc* segs, const SegPlanHdr* hdr, const uint32_t* chunk_seg,
                              size_t max_chunks, const Digits& dg, int passes, uint32_t bins, uint32_t* rows,
                              uint32_t* zero_ptr, size_t zero_words, cudaStream_t s, WsHeader* range_hdr = nullptr) {
    auto kern = k_seg_counts<KeyT, Digits>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)max_count_smem_bytes());
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t grid = std::min<size_t>(max_chunks, (size_t)device_sm_count() * 4);
    KernelScope scope("seg_counts", s);
    kern<<<(unsigned)(grid ? grid : 1), 512, (size_t)passes * bins * 4, s>>>(keys, segs, hdr, chunk_seg, dg, passes,
                                                                            bins, rows, zero_ptr, zero_words,
                                                                            range_hdr);
    return cudaGetLastError();
}

// Device buffers of one segmented sort (all carved from the workspace).
struct SegBuffers {
    WsHeader* ws_hdr;
    SegPlanHdr* hdr;
    SegDesc* large;        // [max_segs]
    SegDesc* small;        // [max_segs]
    SegDesc* tiny;         // [max_segs] segments for the warp sort (null: none)
    uint32_t* tile_seg;    // [max_tiles]
    uint32_t* chunk_seg;   // [max_chunks]
    uint32_t* seg_rows;    // [max_segs][max_passes][max_bins]
    uint32_t* status[2];   // [max_tiles][max_bins] each
    void* tmp_keys;        // [n_total]
    uint32_t* tmp_vals;    // [n_total] or null
    size_t max_segs, max_tiles, max_chunks;
    int max_passes, max_bins;
    int shape;             // segmented pass shape (index into the compiled shapes; 0 = default)
    uint32_t tile_keys;    // keys per tile of that shape (0: the default shape's)
    bool check_range;      // report keys with bits at or above a segment's `bits` in ws_hdr
};

// Workspace layout of a segmented sort: sizes for every region, the offsets
// filled in by carve_seg_buffers.
struct SegLayout {
    size_t off_plan, off_large, off_small, off_tiny, off_tile_seg, off_chunk_seg, off_rows, off_status0, off_status1,
        off_tmp_keys, off_tmp_vals, total;
    size_t max_segs, max_tiles, max_chunks;
    int max_passes, max_bins;
};

SegLayout seg_layout(int key_bytes, bool vals, size_t n_total, size_t max_segs, int max_passes, int max_bins,
                     size_t extra_head);
SegBuffers carve_seg_buffers(void* ws, const SegLayout& L);
uint32_t seg_tile_keys(int key_bytes, bool vals);

// Scatter passes over the large segments already listed in B (their tile and
// chunk ranges reserved, totals in B.hdr): maps, counts, scans and `passes`
// passes of `digit_bits` bits over (key - key_lo).  Pass 0 reads src; pass p
// writes out when (passes-1-p) is even, else the workspace buffer, so the
// last pass lands in out.  src must not be the buffer pass 0 writes.
rs_status enqueue_large_passes(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                               uint32_t* out_v, const SegBuffers& B, int passes, int digit_bits,
                               cudaStream_t stream);

// Same, with the passes' tile counters starting at header slot first_ctr.
rs_status enqueue_large_passes_at(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                                  uint32_t* out_v, const SegBuffers& B, int passes, int digit_bits, int first_ctr,
                                  cudaStream_t stream);

// Bytes of a bucket-sort workspace.
size_t bucket_workspace_bytes(int key_bytes, bool vals, size_t n, size_t nb);

// Shared-memory sorts of a device list of segments (count on the device).
// bucket: device BucketParams for bucket mode, or null.  bucket_table: per
// segment BucketParams indexed by SegDesc::grp (segmented bucket sort; takes
// the place of bucket), with check_range keys outside each segment's [min,
// max] reported.  range_hdr: non-null to report keys at or above 2^bits
// (relative to the segment's key_lo) and, in bucket mode, keys out of range.
rs_status enqueue_local_sorts(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                              uint32_t* out_v, const SegDesc* segs, const uint32_t* count, size_t max_count,
                              const void* bucket, WsHeader* range_hdr, cudaStream_t stream,
                              const void* bucket_table = nullptr, int check_range = 0);

// One array of at most kLocalCap keys sorted in shared memory by a single
// block (a whole radix sort in one launch); keys >= 2^key_bits are reported
// in hdr, whose status word the caller has cleared.  xf: typed-key order.
rs_status enqueue_local_one(int key_bytes, bool vals, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                            uint32_t* vals_out, uint32_t n, int key_bits, WsHeader* hdr, const KeyXform& xf,
                            cudaStream_t stream);

}  // namespace rs
