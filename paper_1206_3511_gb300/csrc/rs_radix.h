// rs_radix.h -- internal interface of the radix-sort host code, shared with
// the bucket-sort, segmented-sort and API translation units.
#pragma once

#include <mutex>

#include "rs_onesweep.cuh"

namespace rs {

// One compiled shape of the scatter-pass kernel.
struct Variant {
    int key_bytes;
    bool vals;
    int block;
    int items;
    int tile_keys;
    cudaError_t (*launch)(const PassParams<RadixDigit>&, cudaStream_t);
    cudaError_t (*launch_typed)(const PassParams<RadixDigit>&, cudaStream_t);  // typed keys; null if not compiled
    size_t (*smem_bytes)(int digit_bits);
};

// Digit width of a radix sort when no kernel shape is requested.
constexpr int kDefaultDigitBits = 8;

// Shared memory a block may use on sm_103a (opt-in maximum).
constexpr size_t kMaxSmemPerBlock = 227 * 1024;

// The largest shared memory a scatter-pass shape needs over the digit widths
// it can run (those whose tables fit in kMaxSmemPerBlock): the value to opt
// the kernel in to.
template <typename Shape>
size_t max_fitting_pass_smem() {
    size_t most = 0;
    for (int D = kMinDigitBits; D <= kMaxDigitBits; ++D)
        if (Shape::smem_bytes(D) <= kMaxSmemPerBlock && Shape::smem_bytes(D) > most) most = Shape::smem_bytes(D);
    return most;
}

// Byte offsets of the regions of a radix-sort workspace.
struct RadixLayout {
    int digit_bits;
    int passes;
    uint32_t bins;
    uint32_t tile_keys;
    uint32_t tiles;
    size_t off_counts, off_scan, off_status[2], off_tmp_keys, off_tmp_vals, total;
};

RadixLayout radix_layout(int key_bytes, bool vals, size_t n, int key_bits, int digit_bits, int tile_keys,
                         bool tmp_buffers);
size_t radix_workspace_bytes(int key_bytes, bool vals, size_t n, int key_bits);
size_t radix_workspace_bytes_cfg(int key_bytes, bool vals, size_t n, int key_bits, const rs_config& cfg);
const Variant* find_variant(int key_bytes, bool vals, int block, int items);
// The shape a sort of n keys takes when none is requested (typed: the key
// mapping is compiled into the first shape of each key type only).
const Variant* default_variant(int key_bytes, bool vals, size_t n, bool typed);

rs_status radix_sort_impl(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                          uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes,
                          cudaStream_t stream, const rs_config* cfg);
// The same for typed keys: digits come from xf.to_ordered(key) (pass 0 maps
// the keys as it loads them, the last pass maps them back as it stores).
rs_status radix_sort_xf(int key_bytes, const void* keys_in, void* keys_out, const uint32_t* vals_in,
                        uint32_t* vals_out, size_t n, int key_bits, void* ws, size_t ws_bytes, cudaStream_t stream,
                        const rs_config* cfg, const KeyXform& xf);

// Checked mode: enqueue the order check of a sort's output (n keys of
// key_bytes bytes at keys) into the status word of hdr.
rs_status enqueue_order_check(int key_bytes, const void* keys, size_t n, const KeyXform& xf, WsHeader* hdr,
                              cudaStream_t stream);

// Grid of the digit-count kernel for n keys.
size_t count_grid(size_t n);

// Launch the digit-count kernel with a digit functor.
template <typename KeyT, typename Digits, bool BYTES>
cudaError_t launch_counts_as(const CountParams& p, const Digits& dg, size_t grid, cudaStream_t s) {
    auto kern = k_digit_counts<KeyT, Digits, BYTES>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)max_count_smem_bytes());
    });
    if (attr_err != cudaSuccess) return attr_err;
    KernelScope scope("digit_counts", s);
    kern<<<(unsigned)grid, kCountBlock, (p.passes * p.bins + kCountBlock / 32 + 1) * 4, s>>>(p, dg);
    return cudaGetLastError();
}

// 8-bit digits from bit 0 take the kernel that reads them as bytes.
template <typename KeyT, typename Digits>
cudaError_t launch_counts(const CountParams& p, const Digits& dg, size_t grid, cudaStream_t s) {
    if constexpr (Digits::kBytesCapable) {
        if (dg.byte_digits()) return launch_counts_as<KeyT, Digits, true>(p, dg, grid, s);
    }
    return launch_counts_as<KeyT, Digits, false>(p, dg, grid, s);
}

// unsorted (nullable): set nonzero if some key is above its successor.
rs_status enqueue_digit_counts(int key_bytes, const void* keys, size_t n, int shift0, int digit_bits, int passes,
                               int key_bits, uint32_t* counts, uint32_t* scan, uint32_t* zero_ptr,
                               size_t zero_words, WsHeader* hdr, cudaStream_t stream,
                               uint32_t* unsorted = nullptr);

}  // namespace rs
