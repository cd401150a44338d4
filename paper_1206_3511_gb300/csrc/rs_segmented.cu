// rs_segmented.cu -- many independent arrays sorted in one call: every
// segment of an offset table is sorted as Algorithm 4 (Sec. 2.5) would sort
// it alone.  Segments of at most kLocalCap keys are sorted inside one block in
// shared memory; larger ones go through per-segment digit counts and
// segmented one-sweep scatter passes.  Planning happens on the device, so a
// call needs no host synchronisation and can be captured in a CUDA graph.
#include <mutex>

#include "rs_bucket.cuh"
#include "rs_segmented.h"

namespace rs {

namespace {

template <typename KeyT, bool VALS, typename BucketFn>
cudaError_t launch_local(const LocalParams& lp, BucketFn bfn, size_t grid, cudaStream_t s) {
    using LS = LocalSmem<KeyT, VALS, kLocalBlock>;
    auto kern = k_local_sort<KeyT, VALS, kLocalBlock, kLocalItems, BucketFn>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    const size_t smem = LS::bytes(kLocalCap);
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr_err != cudaSuccess) return attr_err;
    grid = std::min<size_t>(grid, (size_t)resident_grid(kern, kLocalBlock, smem));
    KernelScope scope("local_sort", s);
    kern<<<(unsigned)(grid ? grid : 1), kLocalBlock, smem, s>>>(lp, bfn);
    return cudaGetLastError();
}

}  // namespace

uint32_t seg_tile_keys(int key_bytes, bool vals) {
    if (key_bytes == 4) return vals ? SegShape<uint32_t, true>::kTile : SegShape<uint32_t, false>::kTile;
    return vals ? SegShape<uint64_t, true>::kTile : SegShape<uint64_t, false>::kTile;
}

namespace {

struct SegVariant {
    int key_bytes;
    bool vals;
    int block, items;
    cudaError_t (*launch)(const SegPassParams<RadixDigit>&, size_t, cudaStream_t);
};

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB>
constexpr SegVariant seg_variant() {
    return SegVariant{(int)sizeof(KeyT), VALS, BLOCK, ITEMS,
                      &launch_seg_pass_shape<KeyT, VALS, BLOCK, ITEMS, MINB, RadixDigit>};
}

// The first entry of each (key width, values) group is SegShape's.
const SegVariant kSegVariants[] = {
    seg_variant<uint32_t, false, 256, 22, 4>(), seg_variant<uint32_t, false, 384, 16, 3>(),
    seg_variant<uint32_t, false, 256, 20, 4>(), seg_variant<uint32_t, false, 256, 24, 4>(),
    seg_variant<uint32_t, false, 256, 26, 4>(), seg_variant<uint32_t, false, 256, 28, 3>(),
    seg_variant<uint32_t, false, 256, 32, 3>(), seg_variant<uint32_t, false, 256, 36, 3>(),
    seg_variant<uint32_t, false, 256, 40, 2>(), seg_variant<uint32_t, false, 384, 24, 2>(),
    seg_variant<uint32_t, false, 512, 20, 2>(),
    seg_variant<uint32_t, false, 256, 18, 4>(),
    seg_variant<uint32_t, false, 256, 15, 4>(), seg_variant<uint32_t, false, 512, 15, 2>(),
    seg_variant<uint32_t, true, 256, 12, 4>(),  seg_variant<uint32_t, true, 256, 15, 3>(),
    seg_variant<uint32_t, true, 256, 18, 3>(),  seg_variant<uint32_t, true, 256, 20, 3>(),
    seg_variant<uint32_t, true, 256, 24, 2>(),
    seg_variant<uint64_t, false, 256, 12, 4>(), seg_variant<uint64_t, false, 256, 9, 4>(),
    seg_variant<uint64_t, false, 384, 12, 3>(), seg_variant<uint64_t, false, 384, 10, 3>(),
    seg_variant<uint64_t, false, 256, 16, 3>(), seg_variant<uint64_t, false, 256, 20, 2>(),
    seg_variant<uint64_t, false, 384, 16, 2>(),
    seg_variant<uint64_t, true, 256, 10, 3>(),  seg_variant<uint64_t, true, 256, 8, 4>(),
    seg_variant<uint64_t, true, 384, 10, 2>(),  seg_variant<uint64_t, true, 384, 8, 3>(),
    seg_variant<uint64_t, true, 256, 12, 3>(),  seg_variant<uint64_t, true, 256, 14, 2>(),
    seg_variant<uint64_t, true, 384, 12, 2>(),
};

const SegVariant* seg_variant_at(int key_bytes, bool vals, int i) {
    for (const SegVariant& v : kSegVariants)
        if (v.key_bytes == key_bytes && v.vals == vals && i-- == 0) return &v;
    return nullptr;
}

}  // namespace

int seg_shape_count(int key_bytes, bool vals) {
    int c = 0;
    for (const SegVariant& v : kSegVariants) c += v.key_bytes == key_bytes && v.vals == vals;
    return c;
}

int seg_shape_find(int key_bytes, bool vals, int block, int items) {
    for (int i = 0; const SegVariant* v = seg_variant_at(key_bytes, vals, i); ++i)
        if (v->block == block && v->items == items) return i;
    return -1;
}

bool seg_shape_get(int key_bytes, bool vals, int i, int* block, int* items) {
    const SegVariant* v = seg_variant_at(key_bytes, vals, i);
    if (!v) return false;
    *block = v->block;
    *items = v->items;
    return true;
}

uint32_t seg_shape_tile(int key_bytes, bool vals, int i) {
    const SegVariant* v = seg_variant_at(key_bytes, vals, i);
    return v ? (uint32_t)(v->block * v->items) : 0u;
}

uint32_t seg_min_tile(int key_bytes, bool vals) {
    uint32_t t = 0;
    for (const SegVariant& v : kSegVariants)
        if (v.key_bytes == key_bytes && v.vals == vals && (t == 0 || (uint32_t)(v.block * v.items) < t))
            t = (uint32_t)(v.block * v.items);
    return t;
}

SegLayout seg_layout(int key_bytes, bool vals, size_t n_total, size_t max_segs, int max_passes, int max_bins,
                     size_t extra_head) {
    SegLayout L{};
    const uint32_t tk = std::min(seg_min_tile(key_bytes, vals), seg_tile_keys(key_bytes, vals));
    L.max_segs = max_segs ? max_segs : 1;
    L.max_tiles = n_total / tk + L.max_segs + 1;
    L.max_chunks = n_total / kSegChunk + L.max_segs + 1;
    L.max_passes = max_passes;
    L.max_bins = max_bins;
    Carver c;
    c.take(sizeof(WsHeader) + extra_head);
    L.off_plan = c.take(sizeof(SegPlanHdr));
    L.off_large = c.take(L.max_segs * sizeof(SegDesc));
    L.off_small = c.take(L.max_segs * sizeof(SegDesc));
    L.off_tiny = c.take(L.max_segs * sizeof(SegDesc));
    L.off_tile_seg = c.take(L.max_tiles * 4);
    L.off_chunk_seg = c.take(L.max_chunks * 4);
    L.off_rows = c.take(L.max_segs * (size_t)max_passes * max_bins * 4);
    L.off_status0 = c.take(L.max_tiles * (size_t)max_bins * 4);
    L.off_status1 = c.take(L.max_tiles * (size_t)max_bins * 4);
    L.off_tmp_keys = c.take(n_total * key_bytes);
    L.off_tmp_vals = vals ? c.take(n_total * 4) : 0;
    L.total = c.off;
    return L;
}

SegBuffers carve_seg_buffers(void* ws, const SegLayout& L) {
    unsigned char* b = static_cast<unsigned char*>(ws);
    SegBuffers B{};
    B.ws_hdr = reinterpret_cast<WsHeader*>(b);
    B.hdr = reinterpret_cast<SegPlanHdr*>(b + L.off_plan);
    B.large = reinterpret_cast<SegDesc*>(b + L.off_large);
    B.small = reinterpret_cast<SegDesc*>(b + L.off_small);
    B.tiny = reinterpret_cast<SegDesc*>(b + L.off_tiny);
    B.tile_seg = reinterpret_cast<uint32_t*>(b + L.off_tile_seg);
    B.chunk_seg = reinterpret_cast<uint32_t*>(b + L.off_chunk_seg);
    B.seg_rows = reinterpret_cast<uint32_t*>(b + L.off_rows);
    B.status[0] = reinterpret_cast<uint32_t*>(b + L.off_status0);
    B.status[1] = reinterpret_cast<uint32_t*>(b + L.off_status1);
    B.tmp_keys = b + L.off_tmp_keys;
    B.tmp_vals = L.off_tmp_vals ? reinterpret_cast<uint32_t*>(b + L.off_tmp_vals) : nullptr;
    B.max_segs = L.max_segs;
    B.max_tiles = L.max_tiles;
    B.max_chunks = L.max_chunks;
    B.max_passes = L.max_passes;
    B.max_bins = L.max_bins;
    return B;
}

template <typename KeyT, bool VALS>
static rs_status large_passes_t(const void* src_k, const uint32_t* src_v, void* out_k, uint32_t* out_v,
                                const SegBuffers& B, int passes, int D, int first_ctr, cudaStream_t stream) {
    const uint32_t bins = 1u << D;
    const uint32_t tk = B.tile_keys ? B.tile_keys : seg_tile_keys(sizeof(KeyT), VALS);
    const SegVariant* var = B.shape ? seg_variant_at(sizeof(KeyT), VALS, B.shape) : nullptr;
    if (B.shape && (!var || (uint32_t)(var->block * var->items) != tk)) return RS_ERR_UNSUPPORTED;
    {
        KernelScope scope("plan_maps", stream);
        k_plan_maps<<<(unsigned)std::min<size_t>(B.max_segs, (size_t)device_sm_count() * 8), 256, 0, stream>>>(
            B.large, B.hdr, tk, B.tile_seg, B.chunk_seg);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    RS_CUDA_TRY(cudaMemsetAsync(B.seg_rows, 0, B.max_segs * (size_t)passes * bins * 4, stream));
    RadixDigits dg{0, D, bins - 1u, 64};
    if (launch_seg_counts<KeyT>(static_cast<const KeyT*>(src_k), B.large, B.hdr, B.chunk_seg, B.max_chunks, dg, passes,
                                bins, B.seg_rows, B.status[0], B.max_tiles * (size_t)bins, stream,
                                B.check_range ? B.ws_hdr : nullptr) != cudaSuccess)
        return RS_ERR_CUDA;
    {
        KernelScope scope("seg_scan", stream);
        k_seg_scan<<<(unsigned)std::min<size_t>(B.max_segs * passes, (size_t)device_sm_count() * 8), 256,
                     (bins + 256 / 32 + 1) * 4, stream>>>(B.seg_rows, B.hdr, passes, bins, 0);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    SegPassParams<RadixDigit> sp{};
    sp.base.digit_bits = D;
    sp.base.hdr = B.ws_hdr;
    sp.base.spin_limit = debug_spin_limit();
    sp.base.stall_tile = debug_stall_tile();
    sp.segs = B.large;
    sp.hdr = B.hdr;
    sp.tile_seg = B.tile_seg;
    sp.seg_base = B.seg_rows;
    sp.passes = passes;
    const void* cur_k = src_k;
    const uint32_t* cur_v = src_v;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        void* dst_k = to_out ? out_k : B.tmp_keys;
        uint32_t* dst_v = VALS ? (to_out ? out_v : B.tmp_vals) : nullptr;
        sp.base.keys_in = cur_k;
        sp.base.keys_out = dst_k;
        sp.base.vals_in = cur_v;
        sp.base.vals_out = dst_v;
        sp.base.op = RadixDigit{p * D, bins - 1u};
        sp.base.status = B.status[p & 1];
        sp.base.status_next = (p + 1 < passes) ? B.status[(p + 1) & 1] : nullptr;
        sp.base.tile_ctr = &B.ws_hdr->tile_ctr[(first_ctr + p) % kMaxPasses];
        sp.pass = p;
        const cudaError_t e = var ? var->launch(sp, B.max_tiles, stream)
                                  : launch_seg_pass<KeyT, VALS, RadixDigit>(sp, B.max_tiles, stream);
        if (e != cudaSuccess) return RS_ERR_CUDA;
        cur_k = dst_k;
        cur_v = dst_v;
    }
    return RS_OK;
}

rs_status enqueue_large_passes_at(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                                  uint32_t* out_v, const SegBuffers& B, int passes, int digit_bits, int first_ctr,
                                  cudaStream_t stream) {
    if (passes < 1 || passes + first_ctr > kMaxPasses || passes > B.max_passes || (1 << digit_bits) > B.max_bins)
        return RS_ERR_INVALID_ARG;
    if (key_bytes == 4)
        return vals ? large_passes_t<uint32_t, true>(src_k, src_v, out_k, out_v, B, passes, digit_bits, first_ctr,
                                                     stream)
                    : large_passes_t<uint32_t, false>(src_k, src_v, out_k, out_v, B, passes, digit_bits, first_ctr,
                                                      stream);
    return vals ? large_passes_t<uint64_t, true>(src_k, src_v, out_k, out_v, B, passes, digit_bits, first_ctr, stream)
                : large_passes_t<uint64_t, false>(src_k, src_v, out_k, out_v, B, passes, digit_bits, first_ctr,
                                                  stream);
}

rs_status enqueue_large_passes(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                               uint32_t* out_v, const SegBuffers& B, int passes, int digit_bits,
                               cudaStream_t stream) {
    return enqueue_large_passes_at(key_bytes, vals, src_k, src_v, out_k, out_v, B, passes, digit_bits, 0, stream);
}

rs_status enqueue_local_sorts(int key_bytes, bool vals, const void* src_k, const uint32_t* src_v, void* out_k,
                              uint32_t* out_v, const SegDesc* segs, const uint32_t* count, size_t max_count,
                              const void* bucket, WsHeader* range_hdr, cudaStream_t stream, const void* bucket_table,
                              int check_range) {
    LocalParams lp{src_k, out_k, src_v, out_v, segs, count, bucket ? bucket : bucket_table, SegDesc{}, range_hdr,
                   KeyXform{}};
    const size_t grid = max_count ? max_count : 1;
    cudaError_t e;
    if (bucket || bucket_table) {
        SegBucketFn f{static_cast<const BucketParams*>(bucket), {}, static_cast<const BucketParams*>(bucket_table),
                      check_range};
        if (key_bytes == 4)
            e = vals ? launch_local<uint32_t, true>(lp, f, grid, stream)
                     : launch_local<uint32_t, false>(lp, f, grid, stream);
        else
            e = vals ? launch_local<uint64_t, true>(lp, f, grid, stream)
                     : launch_local<uint64_t, false>(lp, f, grid, stream);
    } else {
        NoBucket f;
        if (key_bytes == 4)
            e = vals ? launch_local<uint32_t, true>(lp, f, grid, stream)
                     : launch_local<uint32_t, false>(lp, f, grid, stream);
        else
            e = vals ? launch_local<uint64_t, true>(lp, f, grid, stream)
                     : launch_local<uint64_t, false>(lp, f, grid, stream);
    }
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status enqueue_local_one(int key_bytes, bool vals, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                            uint32_t* vals_out, uint32_t n, int key_bits, WsHeader* hdr, const KeyXform& xf,
                            cudaStream_t stream) {
    SegDesc one{};
    one.n = n;
    one.bits = (uint32_t)key_bits;
    LocalParams lp{keys_in, keys_out, vals_in, vals_out, nullptr, nullptr, nullptr, one, hdr, xf};
    NoBucket f;
    cudaError_t e;
    if (key_bytes == 4)
        e = vals ? launch_local<uint32_t, true>(lp, f, 1, stream) : launch_local<uint32_t, false>(lp, f, 1, stream);
    else
        e = vals ? launch_local<uint64_t, true>(lp, f, 1, stream) : launch_local<uint64_t, false>(lp, f, 1, stream);
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

size_t segmented_workspace_bytes(int key_bytes, bool vals, size_t n_total, size_t nseg, int key_bits) {
    const int P = (key_bits + kSegDigitBits - 1) / kSegDigitBits;
    return seg_layout(key_bytes, vals, n_total, nseg, P, 1 << kSegDigitBits, 0).total;
}

static rs_status segmented_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                uint32_t* vals_out, const uint64_t* d_offsets, size_t nseg, size_t n_total,
                                int key_bits, void* ws, size_t ws_bytes, cudaStream_t stream, const rs_config* cfg) {
    const int width = 8 * key_bytes;
    if (key_bits == 0) key_bits = width;
    if (key_bits < 1 || key_bits > width) return RS_ERR_INVALID_ARG;
    if ((vals_in == nullptr) != (vals_out == nullptr)) return RS_ERR_INVALID_ARG;
    const bool vals = vals_in != nullptr;
    if (nseg == 0 || n_total == 0) return RS_OK;
    if (!d_offsets || !keys_in || !keys_out) return RS_ERR_INVALID_ARG;
    if (nseg > ((size_t)1 << 31)) return RS_ERR_INVALID_ARG;
    const size_t kb = n_total * key_bytes, vb = n_total * 4;
    if (keys_in != keys_out && ranges_overlap(keys_in, kb, keys_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && vals_in != vals_out && ranges_overlap(vals_in, vb, vals_out, vb)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)keys_in | (uintptr_t)keys_out) % key_bytes) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    int shape = 0;
    if (cfg) {
        if (cfg->digit_bits != kSegDigitBits) return RS_ERR_UNSUPPORTED;
        shape = seg_shape_find(key_bytes, vals, cfg->block_threads, cfg->items_per_thread);
        if (shape < 0) return RS_ERR_UNSUPPORTED;
    }
    const int D = kSegDigitBits;
    const int P = (key_bits + D - 1) / D;
    const SegLayout L = seg_layout(key_bytes, vals, n_total, nseg, P, 1 << D, 0);
    if (ws_bytes < L.total) return RS_ERR_WORKSPACE;
    SegBuffers B = carve_seg_buffers(ws, L);
    B.shape = shape;
    B.tile_keys = seg_shape_tile(key_bytes, vals, shape);
    B.check_range = true;
    RS_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(B.hdr, 0, sizeof(SegPlanHdr), stream));
    {
        KernelScope scope("plan_segments", stream);
        k_plan_from_offsets<<<(unsigned)((nseg + 255) / 256), 256, 0, stream>>>(
            d_offsets, nseg, (uint64_t)n_total, kLocalCap, B.tile_keys, key_bits, B.large, B.small, B.tiny, B.hdr,
            B.ws_hdr);
        if (cudaGetLastError() != cudaSuccess) return RS_ERR_CUDA;
    }
    // large segments: scatter passes from keys_in (in place with an odd pass
    // count first copies the input to the workspace buffer)
    const void* src_k = keys_in;
    const uint32_t* src_v = vals_in;
    const bool in_place = keys_in == keys_out || (vals && vals_in == vals_out);
    if (in_place && (P % 2 == 1)) {
        RS_CUDA_TRY(cudaMemcpyAsync(B.tmp_keys, keys_in, kb, cudaMemcpyDeviceToDevice, stream));
        src_k = B.tmp_keys;
        if (vals) {
            RS_CUDA_TRY(cudaMemcpyAsync(B.tmp_vals, vals_in, vb, cudaMemcpyDeviceToDevice, stream));
            src_v = B.tmp_vals;
        }
    }
    rs_status st = enqueue_large_passes(key_bytes, vals, src_k, src_v, keys_out, vals_out, B, P, D, stream);
    if (st != RS_OK) return st;
    // small segments: one block each, straight from the input (a block reads
    // its whole segment before writing, so in place is fine)
    st = enqueue_local_sorts(key_bytes, vals, keys_in, vals_in, keys_out, vals_out, B.small, &B.hdr->num_small,
                             nseg, nullptr, B.ws_hdr, stream);
    if (st != RS_OK) return st;
    // tiny segments: one warp each (it too reads a segment before writing it)
    const unsigned grid = (unsigned)std::min<size_t>((nseg + 7) / 8, (size_t)device_sm_count() * 8);
    KernelScope scope("tiny_sort", stream);
    if (key_bytes == 4) {
        if (vals)
            k_tiny_sort<uint32_t, true><<<grid, 256, 0, stream>>>(static_cast<const uint32_t*>(keys_in),
                                                                  static_cast<uint32_t*>(keys_out), vals_in, vals_out,
                                                                  B.tiny, &B.hdr->num_tiny, B.ws_hdr);
        else
            k_tiny_sort<uint32_t, false><<<grid, 256, 0, stream>>>(static_cast<const uint32_t*>(keys_in),
                                                                   static_cast<uint32_t*>(keys_out), nullptr, nullptr,
                                                                   B.tiny, &B.hdr->num_tiny, B.ws_hdr);
    } else {
        if (vals)
            k_tiny_sort<uint64_t, true><<<grid, 256, 0, stream>>>(static_cast<const uint64_t*>(keys_in),
                                                                  static_cast<uint64_t*>(keys_out), vals_in, vals_out,
                                                                  B.tiny, &B.hdr->num_tiny, B.ws_hdr);
        else
            k_tiny_sort<uint64_t, false><<<grid, 256, 0, stream>>>(static_cast<const uint64_t*>(keys_in),
                                                                   static_cast<uint64_t*>(keys_out), nullptr, nullptr,
                                                                   B.tiny, &B.hdr->num_tiny, B.ws_hdr);
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

}  // namespace rs

using namespace rs;

extern "C" {

size_t rs_segmented_workspace_bytes(int key_bytes, int has_values, size_t n_total, size_t nseg, int key_bits) {
    if (key_bytes != 4 && key_bytes != 8) return 0;
    if (key_bits == 0) key_bits = 8 * key_bytes;
    if (key_bits < 1 || key_bits > 8 * key_bytes) return 0;
    return segmented_workspace_bytes(key_bytes, has_values != 0, n_total, nseg, key_bits);
}

rs_status rs_sort_segmented_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return segmented_impl(4, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                          ws_bytes, stream, nullptr);
}

rs_status rs_sort_segmented_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return segmented_impl(8, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                          ws_bytes, stream, nullptr);
}

rs_status rs_sort_segmented_u32_ex(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                                   uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                   int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream, const rs_config* cfg) {
    return segmented_impl(4, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                          ws_bytes, stream, cfg);
}

rs_status rs_sort_segmented_u64_ex(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                                   uint32_t* vals_out, const uint64_t* d_seg_offsets, size_t nseg, size_t n_total,
                                   int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream, const rs_config* cfg) {
    return segmented_impl(8, keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                          ws_bytes, stream, cfg);
}

}  // extern "C"
