// rs_radix.cu -- LSD radix sort (Sec. 2.5, Algorithm 4) on the GPU: one
// digit-count kernel, then ceil(key_bits / D) one-sweep scatter passes that
// ping-pong between keys_out and a workspace buffer and end in keys_out.
#include <algorithm>
#include <mutex>

#include "rs_onesweep.cuh"
#include "rs_radix.h"
#include "rs_segmented.h"

namespace rs {

namespace {

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB, bool XF = false>
cudaError_t launch_pass(const PassParams<RadixDigit>& p, cudaStream_t s) {
    using Shape = OnesweepShape<KeyT, VALS, BLOCK, ITEMS>;
    auto kern = k_onesweep<KeyT, VALS, BLOCK, ITEMS, MINB, RadixDigit, XF>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)max_fitting_pass_smem<Shape>());
    });
    if (attr_err != cudaSuccess) return attr_err;
    const size_t smem = Shape::smem_bytes(p.digit_bits);
    const unsigned grid = (unsigned)std::min<size_t>(p.num_tiles, (size_t)resident_grid(kern, BLOCK, smem));
    KernelScope scope("onesweep_pass", s);
    kern<<<grid ? grid : 1, BLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

using PassLauncher = cudaError_t (*)(const PassParams<RadixDigit>&, cudaStream_t);

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB, bool TYPED>
constexpr PassLauncher typed_launcher() {
    if constexpr (TYPED)
        return &launch_pass<KeyT, VALS, BLOCK, ITEMS, MINB, true>;
    else
        return nullptr;
}

template <typename KeyT, bool VALS, int BLOCK, int ITEMS, int MINB = 1024 / BLOCK, bool TYPED = false>
constexpr Variant make_variant() {
    return Variant{(int)sizeof(KeyT), VALS, BLOCK, ITEMS, BLOCK * ITEMS,
                   &launch_pass<KeyT, VALS, BLOCK, ITEMS, MINB>,
                   typed_launcher<KeyT, VALS, BLOCK, ITEMS, MINB, TYPED>(),
                   &OnesweepShape<KeyT, VALS, BLOCK, ITEMS>::smem_bytes};
}

// Compiled kernel shapes.  The first entry of each (key width, values) group
// is the default, the fastest measured on GB300 at 100M keys with the
// half-warp rank tables and packed ranks:
//   u32 keys only   256 x 36 (3 blocks/SM)  1.57 ms per sort; 256 x 32 1.63,
//                   256 x 26 1.66, 256 x 40 1.72, 256 x 24 1.74, 256 x 22 1.80,
//                   384 x 16 1.91 (larger tiles spread the per-tile work and
//                   shorten the look-back chain, even with 84 bytes spilled)
//   u32 + values    256 x 20 (3 blocks/SM)  2.40 ms; 256 x 18 2.52, 256 x 15 2.78
//   u64 keys only   384 x 16 (2 blocks/SM)  4.89 ms; 384 x 12 5.05, 256 x 16 5.05
//   u64 + values    384 x 12 (2 blocks/SM)  6.60 ms; 256 x 12 6.97, 384 x 10 7.21
// Only the defaults are also compiled for typed keys.
const Variant kVariants[] = {
    make_variant<uint32_t, false, 256, 36, 3, true>(),
    make_variant<uint32_t, false, 256, 22, 4>(),
    make_variant<uint32_t, false, 384, 16, 3>(),
    make_variant<uint32_t, false, 256, 20, 4>(),
    make_variant<uint32_t, false, 256, 24, 4>(),
    make_variant<uint32_t, false, 256, 26, 4>(),
    make_variant<uint32_t, false, 256, 28, 3>(),
    make_variant<uint32_t, false, 256, 32, 3>(),
    make_variant<uint32_t, false, 256, 40, 2>(),
    make_variant<uint32_t, false, 384, 24, 2>(),
    make_variant<uint32_t, false, 512, 20, 2>(),
    make_variant<uint32_t, false, 256, 18, 4>(),
    make_variant<uint32_t, false, 256, 15, 4>(),
    make_variant<uint32_t, false, 512, 15, 2>(),
    make_variant<uint32_t, true, 256, 20, 3, true>(),
    make_variant<uint32_t, true, 256, 15, 3>(),
    make_variant<uint32_t, true, 256, 12, 4>(),
    make_variant<uint32_t, true, 256, 18, 3>(),
    make_variant<uint32_t, true, 256, 24, 2>(),
    make_variant<uint64_t, false, 384, 16, 2, true>(),
    make_variant<uint64_t, false, 384, 12, 3>(),
    make_variant<uint64_t, false, 256, 12, 4>(),
    make_variant<uint64_t, false, 256, 9, 4>(),
    make_variant<uint64_t, false, 384, 10, 3>(),
    make_variant<uint64_t, false, 256, 16, 3>(),
    make_variant<uint64_t, false, 256, 20, 2>(),
    make_variant<uint64_t, true, 384, 12, 2, true>(),
    make_variant<uint64_t, true, 384, 10, 2>(),
    make_variant<uint64_t, true, 256, 10, 3>(),
    make_variant<uint64_t, true, 256, 8, 4>(),
    make_variant<uint64_t, true, 384, 8, 3>(),
    make_variant<uint64_t, true, 256, 12, 3>(),
    make_variant<uint64_t, true, 256, 14, 2>(),
};
// digit widths offered to an autotuner for every kernel shape
constexpr int kTuneDigitBits[] = {8, 4, 5, 6, 7, 9, 10, 11};

}  // namespace

size_t count_grid(size_t n) {
    const size_t chunk = (size_t)kCountBlock * kCountVecIters * 4;
    size_t g = (n + chunk - 1) / chunk;
    size_t cap = (size_t)device_sm_count() * 4;
    if (g > cap) g = cap;
    return g ? g : 1;
}

const Variant* find_variant(int key_bytes, bool vals, int block, int items) {
    for (const Variant& v : kVariants)
        if (v.key_bytes == key_bytes && v.vals == vals && v.block == block && v.items == items) return &v;
    return nullptr;
}

// Up to this many keys an untyped u32 keys-only sort takes the 512 x 15
// shape: with few tiles the look-back chain from tile to tile sets the time,
// and fewer, larger tiles shorten it (79 us against 87 us for 384 x 16 at 1M
// keys, even at 4M; 384 x 16 is faster from 16M keys).
constexpr size_t kSmallSortKeys = (size_t)1 << 22;

const Variant* default_variant(int key_bytes, bool vals, size_t n, bool typed) {
    if (!typed && key_bytes == 4 && !vals && n <= kSmallSortKeys) {
        const Variant* v = find_variant(4, false, 512, 15);
        if (v) return v;
    }
    for (const Variant& v : kVariants)
        if (v.key_bytes == key_bytes && v.vals == vals) return &v;
    return nullptr;
}

int variant_count(int key_bytes, bool vals) {
    int c = 0;
    for (const Variant& v : kVariants) c += (v.key_bytes == key_bytes && v.vals == vals);
    return c;
}

const Variant* variant_at(int key_bytes, bool vals, int i) {
    for (const Variant& v : kVariants)
        if (v.key_bytes == key_bytes && v.vals == vals && i-- == 0) return &v;
    return nullptr;
}

RadixLayout radix_layout(int key_bytes, bool vals, size_t n, int key_bits, int digit_bits, int tile_keys,
                         bool tmp_buffers) {
    RadixLayout L{};
    L.digit_bits = digit_bits;
    L.passes = (key_bits + digit_bits - 1) / digit_bits;
    L.bins = 1u << digit_bits;
    L.tile_keys = (uint32_t)tile_keys;
    L.tiles = (uint32_t)((n + tile_keys - 1) / tile_keys);
    Carver c;
    c.take(sizeof(WsHeader));
    L.off_counts = c.take((size_t)L.passes * L.bins * 4);
    L.off_scan = c.take((size_t)L.passes * L.bins * 4);
    const size_t status_bytes = (size_t)(L.tiles ? L.tiles : 1) * L.bins * 4;
    L.off_status[0] = c.take(status_bytes);
    L.off_status[1] = c.take(status_bytes);
    L.off_tmp_keys = tmp_buffers ? c.take(n * key_bytes) : 0;
    L.off_tmp_vals = (tmp_buffers && vals) ? c.take(n * 4) : 0;
    L.total = c.off;
    return L;
}

size_t radix_workspace_bytes(int key_bytes, bool vals, size_t n, int key_bits) {
    size_t best = 0;
    for (const Variant& v : kVariants) {
        if (v.key_bytes != key_bytes || v.vals != vals) continue;
        for (int D = kMinDigitBits; D <= std::max(kDefaultDigitBits, default_digit_bits()); ++D) {
            size_t t = radix_layout(key_bytes, vals, n, key_bits, D, v.tile_keys, true).total;
            if (t > best) best = t;
        }
    }
    return best;
}

size_t radix_workspace_bytes_cfg(int key_bytes, bool vals, size_t n, int key_bits, const rs_config& cfg) {
    const Variant* v = find_variant(key_bytes, vals, cfg.block_threads, cfg.items_per_thread);
    if (!v) return 0;
    return radix_layout(key_bytes, vals, n, key_bits, cfg.digit_bits, v->tile_keys, true).total;
}

rs_status resolve_config(int key_bytes, bool vals, size_t n, bool typed, const rs_config* cfg, const Variant** var,
                         int* digit_bits) {
    if (!cfg) {
        *var = default_variant(key_bytes, vals, n, typed);
        if (!*var) return RS_ERR_UNSUPPORTED;
        // RS_DIGIT_BITS may ask for wider digits than the default shape's
        // tables allow: then the first compiled shape that holds them (plain
        // keys), else 8-bit digits
        int D = default_digit_bits();
        if ((*var)->smem_bytes(D) > kMaxSmemPerBlock) {
            const Variant* fit = nullptr;
            if (!typed)
                for (const Variant& v : kVariants)
                    if (v.key_bytes == key_bytes && v.vals == vals && v.smem_bytes(D) <= kMaxSmemPerBlock) {
                        fit = &v;
                        break;
                    }
            if (fit)
                *var = fit;
            else
                D = kDefaultDigitBits;
        }
        *digit_bits = D;
        return RS_OK;
    }
    if (cfg->digit_bits < kMinDigitBits || cfg->digit_bits > kMaxDigitBits) return RS_ERR_INVALID_ARG;
    *var = find_variant(key_bytes, vals, cfg->block_threads, cfg->items_per_thread);
    *digit_bits = cfg->digit_bits;
    if (!*var || (*var)->smem_bytes(cfg->digit_bits) > kMaxSmemPerBlock) return RS_ERR_UNSUPPORTED;
    return RS_OK;
}

// Enqueue the digit-count kernel: counts (and their prefixes, if scan != null)
// of `passes` digits starting at bit shift0.  counts must be zero already.
rs_status enqueue_digit_counts(int key_bytes, const void* keys, size_t n, int shift0, int digit_bits, int passes,
                               int key_bits, uint32_t* counts, uint32_t* scan, uint32_t* zero_ptr,
                               size_t zero_words, WsHeader* hdr, cudaStream_t stream, uint32_t* unsorted) {
    CountParams cp{};
    cp.unsorted = unsorted;
    cp.keys = keys;
    cp.n = n;
    cp.passes = passes;
    cp.bins = 1u << digit_bits;
    cp.counts = counts;
    cp.scan = scan;
    cp.zero_ptr = zero_ptr;
    cp.zero_words = zero_words;
    cp.hdr = hdr;
    const RadixDigits dg{shift0, digit_bits, (1u << digit_bits) - 1u, key_bits};
    const size_t grid = count_grid(n);
    cudaError_t e = key_bytes == 4 ? launch_counts<uint32_t>(cp, dg, grid, stream)
                                   : launch_counts<uint64_t>(cp, dg, grid, stream);
    return e == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status radix_sort_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                          uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                          cudaStream_t stream, const rs_config* cfg) {
    return radix_sort_xf(key_bytes, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream, cfg,
                         KeyXform{});
}

rs_status enqueue_order_check(int key_bytes, const void* keys, size_t n, const KeyXform& xf, WsHeader* hdr,
                              cudaStream_t stream) {
    if (n < 2) return RS_OK;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)device_sm_count() * 8);
    KernelScope scope("check_order", stream);
    if (key_bytes == 4)
        k_check_order<uint32_t><<<grid, 256, 0, stream>>>(static_cast<const uint32_t*>(keys), n, xf, hdr);
    else
        k_check_order<uint64_t><<<grid, 256, 0, stream>>>(static_cast<const uint64_t*>(keys), n, xf, hdr);
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

static rs_status radix_sort_xf_body(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                    uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                                    cudaStream_t stream, const rs_config* cfg, const KeyXform& xf);

rs_status radix_sort_xf(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                        uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes, cudaStream_t stream,
                        const rs_config* cfg, const KeyXform& xf) {
    NvtxRange range(key_bytes == 4 ? "rs_sort_u32" : "rs_sort_u64");
    rs_status st = radix_sort_xf_body(key_bytes, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes,
                                      stream, cfg, xf);
    if (st == RS_OK && n > 1 && checked_mode())
        st = enqueue_order_check(key_bytes, keys_out, n, xf, static_cast<WsHeader*>(ws), stream);
    return st;
}

static rs_status radix_sort_xf_body(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                    uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                                    cudaStream_t stream, const rs_config* cfg, const KeyXform& xf) {
    const int width = 8 * key_bytes;
    if (key_bits == 0) key_bits = width;
    if (key_bits < 1 || key_bits > width) return RS_ERR_INVALID_ARG;
    if (xf.active() && key_bits != width) return RS_ERR_INVALID_ARG;  // typed keys use every bit
    if (xf.active() && cfg) return RS_ERR_UNSUPPORTED;                 // typed kernels: default shapes only
    if ((vals_in == nullptr) != (vals_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS) return RS_ERR_INVALID_ARG;
    const bool vals = vals_in != nullptr;
    const Variant* var = nullptr;
    int D = 0;
    rs_status st = resolve_config(key_bytes, vals, n, xf.active(), cfg, &var, &D);
    if (st != RS_OK) return st;
    if (n == 0) return RS_OK;
    if (!keys_in || !keys_out) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)keys_in | (uintptr_t)keys_out) % key_bytes) return RS_ERR_INVALID_ARG;
    if (vals && (((uintptr_t)vals_in | (uintptr_t)vals_out) % 4)) return RS_ERR_INVALID_ARG;
    const size_t kb = n * key_bytes, vb = n * 4;
    if (keys_in != keys_out && ranges_overlap(keys_in, kb, keys_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && vals_in != vals_out && ranges_overlap(vals_in, vb, vals_out, vb)) return RS_ERR_INVALID_ARG;
    if (vals && (ranges_overlap(keys_out, kb, vals_out, vb) || ranges_overlap(keys_in, kb, vals_out, vb)))
        return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;

    const RadixLayout L = radix_layout(key_bytes, vals, n, key_bits, D, var->tile_keys, true);
    if (ws_bytes < L.total) return RS_ERR_WORKSPACE;
    if (ranges_overlap(ws, L.total, keys_out, kb) || ranges_overlap(ws, L.total, keys_in, kb))
        return RS_ERR_INVALID_ARG;
    unsigned char* base = static_cast<unsigned char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.off_counts);
    uint32_t* scan = reinterpret_cast<uint32_t*>(base + L.off_scan);
    uint32_t* status[2] = {reinterpret_cast<uint32_t*>(base + L.off_status[0]),
                           reinterpret_cast<uint32_t*>(base + L.off_status[1])};
    void* tmpk = base + L.off_tmp_keys;
    uint32_t* tmpv = vals ? reinterpret_cast<uint32_t*>(base + L.off_tmp_vals) : nullptr;

    // zero the per-call part of the header and the counts
    RS_CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(WsHeader), stream));
    // a small array without a requested kernel shape is sorted whole by one
    // block in shared memory: one launch instead of a count and P passes
    if (!cfg && n <= kLocalCap)
        return enqueue_local_one(key_bytes, vals, keys_in, vals_in, keys_out, vals_out, (uint32_t)n, key_bits, hdr,
                                 xf, stream);
    RS_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)L.passes * L.bins * 4, stream));

    const int P = L.passes;
    // ping-pong: pass p writes keys_out when (P-1-p) is even, so the last
    // pass lands in keys_out.  In place with P odd would make pass 0 write the
    // array it reads, so the input is first copied to the workspace buffer.
    const bool in_place = keys_in == keys_out || (vals && vals_in == vals_out);
    const void* src_k = keys_in;
    const uint32_t* src_v = vals_in;
    if (in_place && (P % 2 == 1)) {
        RS_CUDA_TRY(cudaMemcpyAsync(tmpk, keys_in, kb, cudaMemcpyDeviceToDevice, stream));
        src_k = tmpk;
        if (vals) {
            RS_CUDA_TRY(cudaMemcpyAsync(tmpv, vals_in, vb, cudaMemcpyDeviceToDevice, stream));
            src_v = tmpv;
        }
    }
    const size_t status_words = (size_t)L.tiles * L.bins;
    uint32_t* unsorted = &hdr->unsorted;  // the count kernel checks whether the input is already in order
    if (xf.active()) {
        CountParams cp{src_k, n, P, L.bins, counts, scan, status[0], status_words, hdr, unsorted};
        const OrderedRadixDigits dg{RadixDigits{0, D, L.bins - 1u, key_bits}, xf};
        const cudaError_t e = key_bytes == 4 ? launch_counts<uint32_t>(cp, dg, count_grid(n), stream)
                                             : launch_counts<uint64_t>(cp, dg, count_grid(n), stream);
        if (e != cudaSuccess) return RS_ERR_CUDA;
    } else {
        st = enqueue_digit_counts(key_bytes, src_k, n, 0, D, P, key_bits, counts, scan, status[0], status_words, hdr,
                                  stream, unsorted);
        if (st != RS_OK) return st;
    }

    PassParams<RadixDigit> pp{};
    pp.n = (uint32_t)n;
    pp.num_tiles = L.tiles;
    pp.digit_bits = D;
    pp.hdr = hdr;
    pp.spin_limit = debug_spin_limit();
    pp.stall_tile = debug_stall_tile();
    for (int p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p) % 2) == 0;
        void* dst_k = to_out ? keys_out : tmpk;
        uint32_t* dst_v = vals ? (to_out ? vals_out : tmpv) : nullptr;
        pp.keys_in = src_k;
        pp.keys_out = dst_k;
        pp.vals_in = src_v;
        pp.vals_out = dst_v;
        // the last pass ranks only the key bits left (20-bit keys: 8 + 8 + 4),
        // so its tables, scan and look-back cover 2^w digits, not 2^D
        const int w = std::min(D, key_bits - p * D);
        pp.digit_bits = w;
        pp.op = RadixDigit{p * D, (1u << w) - 1u};
        pp.digit_base = scan + (size_t)p * L.bins;
        pp.status = status[p & 1];
        pp.status_next = (p + 1 < P) ? status[(p + 1) & 1] : nullptr;
        pp.tile_ctr = &hdr->tile_ctr[p];
        pp.xf = xf;
        pp.xf_in = xf.active() && p == 0;
        pp.xf_out = xf.active() && p == P - 1;
        cudaError_t e = xf.active() ? var->launch_typed(pp, stream) : var->launch(pp, stream);
        if (e != cudaSuccess) return RS_ERR_CUDA;
        src_k = dst_k;
        src_v = dst_v;
    }
    return RS_OK;
}

rs_status counting_pass_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                             uint32_t* vals_out, size_t n, int shift, int digit_bits, void* ws, size_t ws_bytes,
                             cudaStream_t stream) {
    const int width = 8 * key_bytes;
    if (digit_bits < kMinDigitBits || digit_bits > kMaxDigitBits) return RS_ERR_INVALID_ARG;
    if (shift < 0 || shift >= width) return RS_ERR_INVALID_ARG;
    if ((vals_in == nullptr) != (vals_out == nullptr)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS) return RS_ERR_INVALID_ARG;
    const bool vals = vals_in != nullptr;
    if (n == 0) return RS_OK;
    if (!keys_in || !keys_out) return RS_ERR_INVALID_ARG;
    const size_t kb = n * key_bytes, vb = n * 4;
    if (ranges_overlap(keys_in, kb, keys_out, kb)) return RS_ERR_INVALID_ARG;
    if (vals && ranges_overlap(vals_in, vb, vals_out, vb)) return RS_ERR_INVALID_ARG;
    if (((uintptr_t)keys_in | (uintptr_t)keys_out) % key_bytes) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    // the default shape, or the first that fits this digit width's tables
    const Variant* var = default_variant(key_bytes, vals, n, false);
    if (var && var->smem_bytes(digit_bits) > kMaxSmemPerBlock) {
        var = nullptr;
        for (const Variant& v : kVariants)
            if (v.key_bytes == key_bytes && v.vals == vals && v.smem_bytes(digit_bits) <= kMaxSmemPerBlock) {
                var = &v;
                break;
            }
    }
    if (!var) return RS_ERR_UNSUPPORTED;
    const RadixLayout L = radix_layout(key_bytes, vals, n, digit_bits, digit_bits, var->tile_keys, false);
    if (ws_bytes < L.total) return RS_ERR_WORKSPACE;
    unsigned char* base = static_cast<unsigned char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + L.off_counts);
    uint32_t* scan = reinterpret_cast<uint32_t*>(base + L.off_scan);
    uint32_t* status = reinterpret_cast<uint32_t*>(base + L.off_status[0]);
    RS_CUDA_TRY(cudaMemsetAsync(base, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)L.bins * 4, stream));
    rs_status st = enqueue_digit_counts(key_bytes, keys_in, n, shift, digit_bits, 1, width, counts, scan, status,
                                        (size_t)L.tiles * L.bins, hdr, stream);
    if (st != RS_OK) return st;
    PassParams<RadixDigit> pp{};
    pp.keys_in = keys_in;
    pp.keys_out = keys_out;
    pp.vals_in = vals_in;
    pp.vals_out = vals_out;
    pp.n = (uint32_t)n;
    pp.num_tiles = L.tiles;
    pp.digit_bits = digit_bits;
    pp.op = RadixDigit{shift, L.bins - 1u};
    pp.digit_base = scan;
    pp.status = status;
    pp.status_next = nullptr;
    pp.tile_ctr = &hdr->tile_ctr[0];
    pp.hdr = hdr;
    pp.spin_limit = debug_spin_limit();
    pp.stall_tile = debug_stall_tile();
    return var->launch(pp, stream) == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

rs_status digit_counts_impl(int key_bytes, const void* keys, size_t n, int key_bits, int digit_bits,
                            uint32_t* counts_out, void* ws, size_t ws_bytes, cudaStream_t stream) {
    const int width = 8 * key_bytes;
    if (key_bits == 0) key_bits = width;
    if (key_bits < 1 || key_bits > width) return RS_ERR_INVALID_ARG;
    if (digit_bits < kMinDigitBits || digit_bits > kMaxDigitBits) return RS_ERR_INVALID_ARG;
    if (!counts_out || ((uintptr_t)counts_out % 4)) return RS_ERR_INVALID_ARG;
    if (n > RS_MAX_KEYS) return RS_ERR_INVALID_ARG;
    if (n && !keys) return RS_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256)) return RS_ERR_WORKSPACE;
    if (ws_bytes < sizeof(WsHeader)) return RS_ERR_WORKSPACE;
    const int P = (key_bits + digit_bits - 1) / digit_bits;
    WsHeader* hdr = static_cast<WsHeader*>(ws);
    RS_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(WsHeader), stream));
    RS_CUDA_TRY(cudaMemsetAsync(counts_out, 0, (size_t)P * ((size_t)1 << digit_bits) * 4, stream));
    if (n == 0) return RS_OK;
    return enqueue_digit_counts(key_bytes, keys, n, 0, digit_bits, P, key_bits, counts_out, nullptr, nullptr, 0,
                                hdr, stream);
}

}  // namespace rs

using namespace rs;

extern "C" {

rs_status rs_sort_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      size_t n, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return radix_sort_impl(4, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream, nullptr);
}

rs_status rs_sort_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                      size_t n, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream) {
    return radix_sort_impl(8, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream, nullptr);
}

rs_status rs_sort_typed(int key_kind, int key_bytes, int descending, const void* keys_in, void* keys_out,
                        const uint32_t* vals_in, uint32_t* vals_out, size_t n, void* ws, size_t ws_bytes,
                        rs_stream_t stream) {
    if (key_kind != RS_KEY_UINT && key_kind != RS_KEY_INT && key_kind != RS_KEY_FLOAT) return RS_ERR_INVALID_ARG;
    if (key_bytes != 4 && key_bytes != 8) return RS_ERR_INVALID_ARG;
    const KeyXform xf{key_kind == RS_KEY_INT ? kKindSigned : key_kind == RS_KEY_FLOAT ? kKindFloat : kKindUnsigned,
                      descending ? 1 : 0};
    return radix_sort_xf(key_bytes, keys_in, keys_out, vals_in, vals_out, n, 0, ws, ws_bytes, stream, nullptr, xf);
}

rs_status rs_sort_u32_ex(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         size_t n, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream,
                         const rs_config* cfg) {
    return radix_sort_impl(4, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream, cfg);
}

rs_status rs_sort_u64_ex(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         size_t n, int key_bits, void* ws, size_t ws_bytes, rs_stream_t stream,
                         const rs_config* cfg) {
    return radix_sort_impl(8, keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream, cfg);
}

rs_status rs_digit_counts_u32(const uint32_t* keys, size_t n, int key_bits, int digit_bits, uint32_t* counts_out,
                              void* ws, size_t ws_bytes, rs_stream_t stream) {
    return digit_counts_impl(4, keys, n, key_bits, digit_bits, counts_out, ws, ws_bytes, stream);
}

rs_status rs_digit_counts_u64(const uint64_t* keys, size_t n, int key_bits, int digit_bits, uint32_t* counts_out,
                              void* ws, size_t ws_bytes, rs_stream_t stream) {
    return digit_counts_impl(8, keys, n, key_bits, digit_bits, counts_out, ws, ws_bytes, stream);
}

rs_status rs_counting_pass_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in,
                               uint32_t* vals_out, size_t n, int shift, int digit_bits, void* ws, size_t ws_bytes,
                               rs_stream_t stream) {
    return counting_pass_impl(4, keys_in, keys_out, vals_in, vals_out, n, shift, digit_bits, ws, ws_bytes, stream);
}

rs_status rs_counting_pass_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in,
                               uint32_t* vals_out, size_t n, int shift, int digit_bits, void* ws, size_t ws_bytes,
                               rs_stream_t stream) {
    return counting_pass_impl(8, keys_in, keys_out, vals_in, vals_out, n, shift, digit_bits, ws, ws_bytes, stream);
}

rs_status rs_default_config(int key_bytes, int has_values, size_t n, rs_config* out) {
    if ((key_bytes != 4 && key_bytes != 8) || !out) return RS_ERR_INVALID_ARG;
    const Variant* v = nullptr;
    int D = 0;
    if (resolve_config(key_bytes, has_values != 0, n, false, nullptr, &v, &D) != RS_OK) return RS_ERR_UNSUPPORTED;
    out->digit_bits = D;
    out->block_threads = v->block;
    out->items_per_thread = v->items;
    return RS_OK;
}

int rs_config_count(int key_bytes, int has_values) {
    if (key_bytes != 4 && key_bytes != 8) return 0;
    int c = 0;
    for (int vi = 0; vi < variant_count(key_bytes, has_values != 0); ++vi) {
        const Variant* v = variant_at(key_bytes, has_values != 0, vi);
        for (int D : kTuneDigitBits) c += v->smem_bytes(D) <= kMaxSmemPerBlock;
    }
    return c;
}

rs_status rs_config_get(int key_bytes, int has_values, int i, rs_config* out) {
    if ((key_bytes != 4 && key_bytes != 8) || !out || i < 0) return RS_ERR_INVALID_ARG;
    for (int vi = 0; vi < variant_count(key_bytes, has_values != 0); ++vi) {
        const Variant* v = variant_at(key_bytes, has_values != 0, vi);
        for (int D : kTuneDigitBits) {
            if (v->smem_bytes(D) > kMaxSmemPerBlock) continue;
            if (i-- == 0) {
                out->digit_bits = D;
                out->block_threads = v->block;
                out->items_per_thread = v->items;
                return RS_OK;
            }
        }
    }
    return RS_ERR_INVALID_ARG;
}

}  // extern "C"
