"""GB300 (sm_103a) integer sorts: LSD radix sort and bucket sort after
Horsmalahti, "Comparison of Bucket Sort and RADIX Sort" (arXiv:1206.3511).

Every step runs in hand-written CUDA kernels inside librsort.so, reached
through its C ABI (include/rsort.h).  PyTorch provides device memory and
streams only.  The low-level functions of ``_lib`` carry the C names
(``rs_sort_u32`` ...); the helpers below allocate outputs and workspaces with
torch and raise ``SortError`` on a non-zero status.

Keys are unsigned integers.  torch tensors of dtype uint32/int32 are treated as
32-bit keys and uint64/int64 as 64-bit keys, bit for bit (a signed tensor's
bits are sorted as unsigned).  Values are 32-bit (uint32 or int32).
"""
from __future__ import annotations

from . import _lib
from ._lib import (bs_segmented_workspace_bytes, bs_sort_segmented_u32, bs_sort_segmented_u64,
                   rs_sort_segmented_u32_ex, rs_sort_segmented_u64_ex, rs_server_release, bs_bucket_counts_u32, bs_bucket_counts_u64, RS_KEY_FLOAT, RS_KEY_INT, RS_KEY_UINT, rs_sort_typed, RS_PLAN_BUCKET, RS_PLAN_RADIX, RS_PLAN_SEGMENTED, RsPlanDesc, rs_plan_create, rs_plan_destroy,
                   rs_plan_info, rs_plan_launch, RsRequest, RsResult, RsServerConfig, RsServerStats, rs_server_create, rs_server_destroy,
                   rs_server_get_stats, rs_server_poll, rs_server_submit, rs_server_wait, bs_sort_u32, bs_sort_u64, rs_segmented_workspace_bytes, rs_sort_segmented_u32, rs_sort_segmented_u64,
                   RS_ALGO_BUCKET, RS_ALGO_RADIX, STATUS, RsConfig, load, rs_config_count, rs_config_get,
                   rs_counting_pass_u32, rs_counting_pass_u64, rs_default_config, rs_digit_counts_u32,
                   rs_digit_counts_u64, rs_get_status, rs_launch_count, rs_profile_enable, rs_profile_read,
                   rs_set_debug, rs_sort_u32, rs_sort_u32_ex, rs_sort_u32_noalloc, rs_sort_u64,
                   rs_host_sort_bytes, rs_sort_host_u32, rs_sort_host_u64, bs_sort_host_u32, bs_sort_host_u64,
                   rs_segmented_host_bytes, rs_sort_segmented_host_u32, rs_sort_segmented_host_u64,
                   rs_sort_u64_ex, rs_status_string, rs_version, rs_workspace_bytes, rs_workspace_bytes_cfg)

__all__ = [
    "SortError", "load", "sort", "counting_pass", "digit_counts", "workspace", "get_status", "key_bytes_of",
    "rs_sort_u32", "rs_sort_u64", "rs_sort_u32_ex", "rs_sort_u64_ex", "rs_digit_counts_u32", "rs_digit_counts_u64",
    "rs_counting_pass_u32", "rs_counting_pass_u64", "rs_get_status", "rs_set_debug", "rs_status_string",
    "rs_version", "rs_workspace_bytes", "rs_workspace_bytes_cfg", "rs_default_config", "rs_config_count",
    "rs_config_get", "RsConfig", "RS_ALGO_RADIX", "RS_ALGO_BUCKET", "STATUS", "rs_profile_enable",
    "rs_profile_read", "rs_launch_count", "rs_sort_u32_noalloc", "rs_segmented_workspace_bytes",
    "rs_sort_segmented_u32", "rs_sort_segmented_u64", "segmented_sort", "bs_sort_u32", "bs_sort_u64",
    "bucket_sort", "Server", "Plan", "sort_typed", "rs_sort_typed", "bs_bucket_counts_u32", "bs_bucket_counts_u64",
    "RS_KEY_UINT", "RS_KEY_INT", "RS_KEY_FLOAT", "RsPlanDesc", "rs_plan_create", "rs_plan_destroy", "rs_plan_info",
    "rs_plan_launch", "RS_PLAN_RADIX", "RS_PLAN_BUCKET", "RS_PLAN_SEGMENTED", "RsRequest", "RsResult",
    "RsServerConfig", "RsServerStats", "rs_server_create", "rs_server_destroy", "rs_server_get_stats",
    "rs_server_poll", "rs_server_submit", "rs_server_wait", "rs_server_release", "rs_sort_segmented_u32_ex",
    "rs_sort_segmented_u64_ex", "rs_host_sort_bytes", "rs_sort_host_u32", "rs_sort_host_u64", "sort_host",
    "bs_sort_host_u32", "bs_sort_host_u64", "rs_segmented_host_bytes", "rs_sort_segmented_host_u32",
    "rs_sort_segmented_host_u64", "bs_segmented_workspace_bytes", "bs_sort_segmented_u32", "bs_sort_segmented_u64",
    "segmented_bucket_sort",
]


class SortError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}" if what else STATUS.get(code, str(code)))


def check(code: int, what: str = "") -> None:
    if code != 0:
        raise SortError(code, what)


def key_bytes_of(t) -> int:
    import torch

    if t.dtype in (torch.uint32, torch.int32):
        return 4
    if t.dtype in (torch.uint64, torch.int64):
        return 8
    raise TypeError(f"keys must be a 32- or 64-bit integer tensor, got {t.dtype}")


def _check_tensor(t, what):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def workspace(nbytes: int, device=None):
    """A uint8 device buffer of nbytes (torch's allocator aligns it to >= 256 B)."""
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def sort(keys, values=None, key_bits: int = 0, out=None, out_values=None, ws=None, stream=None, config=None):
    """Stable LSD radix sort of a 1-D CUDA tensor (rs_sort_u32 / rs_sort_u64).
    Returns (sorted_keys, sorted_values or None)."""
    import torch

    _check_tensor(keys, "keys")
    kb = key_bytes_of(keys)
    n = keys.numel()
    if values is not None:
        _check_tensor(values, "values")
        if values.numel() != n or values.element_size() != 4:
            raise ValueError("values must be 32-bit with one entry per key")
    out = torch.empty_like(keys) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values)
    cfg = _lib._as_cfg(config)
    if ws is None:
        if cfg is not None:
            nbytes = rs_workspace_bytes_cfg(kb, values is not None, n, key_bits, cfg)
        else:
            nbytes = rs_workspace_bytes(RS_ALGO_RADIX, kb, values is not None, n, key_bits, 0, out is keys)
        ws = workspace(nbytes, keys.device)
    fn = rs_sort_u32_ex if kb == 4 else rs_sort_u64_ex
    check(fn(keys, out, values, out_values, n, key_bits, ws, ws.numel(), stream, cfg), "rs_sort")
    return out, out_values


def sort_host(keys, values=None, key_bits: int = 0, out=None, out_values=None, dev_buf=None, stream=None,
              algo: int = RS_ALGO_RADIX, min_key=None, max_key=None, num_buckets: int = 0):
    """Sort a 1-D CPU tensor on the GPU through the host-buffer calls:
    rs_sort_host_* for algo RS_ALGO_RADIX, bs_sort_host_* for RS_ALGO_BUCKET
    (bounds and bucket count as in bucket_sort).  Copy in, sort and copy out
    are all enqueued on `stream`.  Returns (sorted_keys, sorted_values or
    None) as CPU tensors; with pinned tensors the copies are asynchronous and
    the results are ready once `stream` has passed the call."""
    import torch

    if keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CPU tensor")
    kb = key_bytes_of(keys)
    n = keys.numel()
    if values is not None:
        if values.is_cuda or not values.is_contiguous() or values.numel() != n or values.element_size() != 4:
            raise ValueError("values must be a contiguous 32-bit CPU tensor with one entry per key")
    out = torch.empty_like(keys, pin_memory=keys.is_pinned()) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values, pin_memory=values.is_pinned())
    if dev_buf is None:
        dev_buf = workspace(rs_host_sort_bytes(algo, kb, values is not None, n, key_bits, num_buckets))
    if algo == RS_ALGO_RADIX:
        fn = rs_sort_host_u32 if kb == 4 else rs_sort_host_u64
        rc = fn(keys, out, values, out_values, n, key_bits, dev_buf, dev_buf.numel(), stream)
    else:
        if (min_key is None) != (max_key is None):
            raise ValueError("give both min_key and max_key, or neither")
        if min_key is None:
            min_key, max_key = (1, 0)  # min > max: bounds from the data
        fn = bs_sort_host_u32 if kb == 4 else bs_sort_host_u64
        rc = fn(keys, out, values, out_values, n, min_key, max_key, num_buckets, dev_buf, dev_buf.numel(), stream)
    check(rc, "sort_host")
    return out, out_values


def counting_pass(keys, values=None, shift: int = 0, digit_bits: int = 8, ws=None, stream=None):
    """One stable counting-sort pass on digit (key >> shift) & (2^digit_bits - 1)."""
    import torch

    _check_tensor(keys, "keys")
    kb = key_bytes_of(keys)
    n = keys.numel()
    out = torch.empty_like(keys)
    out_values = torch.empty_like(values) if values is not None else None
    if ws is None:
        ws = workspace(rs_workspace_bytes(RS_ALGO_RADIX, kb, values is not None, n, 0, 0, 0), keys.device)
    fn = rs_counting_pass_u32 if kb == 4 else rs_counting_pass_u64
    check(fn(keys, out, values, out_values, n, shift, digit_bits, ws, ws.numel(), stream), "rs_counting_pass")
    return out, out_values


def digit_counts(keys, key_bits: int = 0, digit_bits: int = 8, ws=None, stream=None):
    """Per-pass digit counts, shape (ceil(key_bits/D), 2^D), as an int64 tensor."""
    import torch

    _check_tensor(keys, "keys")
    kb = key_bytes_of(keys)
    kbits = key_bits or 8 * kb
    P = (kbits + digit_bits - 1) // digit_bits
    counts = torch.empty(P * (1 << digit_bits), dtype=torch.int32, device=keys.device)
    if ws is None:
        ws = workspace(256, keys.device)
    fn = rs_digit_counts_u32 if kb == 4 else rs_digit_counts_u64
    check(fn(keys, keys.numel(), key_bits, digit_bits, counts, ws, ws.numel(), stream), "rs_digit_counts")
    return counts.view(P, 1 << digit_bits).to(torch.int64)


_TYPED = {"int32": (1, 4), "int64": (1, 8), "float32": (2, 4), "float64": (2, 8)}


def sort_typed(keys, values=None, kind=None, descending: bool = False, out=None, out_values=None, ws=None,
               stream=None):
    """Stable radix sort of signed or floating-point keys, ascending or
    descending (rs_sort_typed).  kind: RS_KEY_UINT / RS_KEY_INT / RS_KEY_FLOAT,
    or None to take it from the tensor dtype (int32/int64 signed, float32/
    float64 float).  Floats are ordered by IEEE-754 totalOrder.  Returns
    (keys, values or None)."""
    import torch

    _check_tensor(keys, "keys")
    name = str(keys.dtype).replace("torch.", "")
    if kind is None:
        if name not in _TYPED:
            raise ValueError(f"no key kind for dtype {keys.dtype}")
        kind = _TYPED[name][0]
    kb = keys.element_size()
    if kb not in (4, 8):
        raise ValueError("keys must be 4 or 8 bytes wide")
    n = keys.numel()
    out = torch.empty_like(keys) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values)
    if ws is None:
        ws = workspace(rs_workspace_bytes(RS_ALGO_RADIX, kb, values is not None, n, 0, 0, out is keys), keys.device)
    check(rs_sort_typed(kind, kb, descending, keys, out, values, out_values, n, ws, ws.numel(), stream),
          "rs_sort_typed")
    return out, out_values


def get_status(ws, stream=None) -> int:
    """Read and clear the device status word of a workspace (syncs the stream)."""
    return rs_get_status(ws, stream)


def segmented_sort(keys, offsets, values=None, key_bits: int = 0, out=None, out_values=None, ws=None, stream=None):
    """Sort every segment [offsets[s], offsets[s+1]) of a 1-D CUDA tensor on
    its own (rs_sort_segmented_u32/u64).  offsets: int64/uint64 CUDA tensor of
    nseg+1 entries.  Returns (keys, values or None)."""
    import torch

    _check_tensor(keys, "keys")
    _check_tensor(offsets, "offsets")
    kb = key_bytes_of(keys)
    n = keys.numel()
    nseg = offsets.numel() - 1
    out = torch.empty_like(keys) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values)
    if ws is None:
        ws = workspace(rs_segmented_workspace_bytes(kb, values is not None, n, max(nseg, 1), key_bits), keys.device)
    fn = rs_sort_segmented_u32 if kb == 4 else rs_sort_segmented_u64
    check(fn(keys, out, values, out_values, offsets, nseg, n, key_bits, ws, ws.numel(), stream), "rs_sort_segmented")
    return out, out_values


def segmented_bucket_sort(keys, offsets, values=None, min_key=None, max_key=None, keys_per_bucket: int = 0, out=None,
                          out_values=None, ws=None, stream=None):
    """Bucket-sort every segment [offsets[s], offsets[s+1]) of a 1-D CUDA
    tensor on its own (bs_sort_segmented_u32/u64).  min_key/max_key: bounds
    declared for every segment (both None: each segment's own, found on the
    device).  keys_per_bucket 0 means 16.  Returns (keys, values or None)."""
    import torch

    _check_tensor(keys, "keys")
    _check_tensor(offsets, "offsets")
    kb = key_bytes_of(keys)
    n = keys.numel()
    nseg = offsets.numel() - 1
    out = torch.empty_like(keys) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values)
    if ws is None:
        ws = workspace(bs_segmented_workspace_bytes(kb, values is not None, n, max(nseg, 1), keys_per_bucket),
                       keys.device)
    lo, hi = (1, 0) if min_key is None else (min_key, max_key)
    fn = bs_sort_segmented_u32 if kb == 4 else bs_sort_segmented_u64
    check(fn(keys, out, values, out_values, offsets, nseg, n, lo, hi, keys_per_bucket, ws, ws.numel(), stream),
          "bs_sort_segmented")
    return out, out_values


def bucket_sort(keys, values=None, min_key=None, max_key=None, num_buckets: int = 0, out=None, out_values=None,
                ws=None, stream=None):
    """Stable bucket sort (bs_sort_u32 / bs_sort_u64).  min_key/max_key: the
    declared key range (both None: computed on the device).  num_buckets 0
    means max(1, n // 16).  Returns (keys, values or None)."""
    import torch

    _check_tensor(keys, "keys")
    kb = key_bytes_of(keys)
    n = keys.numel()
    if (min_key is None) != (max_key is None):
        raise ValueError("give both min_key and max_key, or neither")
    if min_key is None:
        min_key, max_key = (1, 0)  # min > max: bounds from the data
    out = torch.empty_like(keys) if out is None else out
    if values is not None and out_values is None:
        out_values = torch.empty_like(values)
    if ws is None:
        ws = workspace(rs_workspace_bytes(RS_ALGO_BUCKET, kb, values is not None, n, 0, num_buckets, out is keys),
                       keys.device)
    fn = bs_sort_u32 if kb == 4 else bs_sort_u64
    check(fn(keys, out, values, out_values, n, min_key, max_key, num_buckets, ws, ws.numel(), stream), "bs_sort")
    return out, out_values


class Server:
    """Sort server over the C ABI (rs_server_*): requests are sorted
    asynchronously with admission under a memory budget and continuous
    batching.  The device pool is a torch uint8 buffer kept alive here."""

    def __init__(self, pool_bytes: int, budget_bytes: int = 0, num_streams: int = 4, max_batch: int = 64,
                 batch_max_keys: int = 0, device=None):
        self.pool = workspace(pool_bytes, device)
        cfg = RsServerConfig(self.pool.data_ptr(), self.pool.numel(), budget_bytes, num_streams, max_batch,
                             batch_max_keys)
        rc, self.handle = rs_server_create(cfg)
        check(rc, "rs_server_create")
        self._keep = {}

    def submit(self, keys_in, keys_out, vals_in=None, vals_out=None, algo: int = RS_ALGO_RADIX, key_bits: int = 0,
               min_key: int = 1, max_key: int = 0, num_buckets: int = 0) -> int:
        """Queue one sort; returns its ticket.  The tensors must stay alive
        and untouched until the request is done (kept referenced here)."""
        req = RsRequest(algo, key_bytes_of(keys_in), keys_in.data_ptr(), keys_out.data_ptr(),
                        vals_in.data_ptr() if vals_in is not None else None,
                        vals_out.data_ptr() if vals_out is not None else None, keys_in.numel(), key_bits,
                        min_key, max_key, num_buckets)
        rc, ticket = rs_server_submit(self.handle, req)
        check(rc, "rs_server_submit")
        self._keep[ticket] = (keys_in, keys_out, vals_in, vals_out)
        return ticket

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        rc = rs_server_wait(self.handle, ticket, timeout_ms)
        if rc != 7:  # done (RS_ERR_NOT_READY means still running)
            self._keep.pop(ticket, None)
        return rc

    def result(self, ticket: int):
        return rs_server_poll(self.handle, ticket)

    def release(self, ticket: int) -> int:
        """Forget a finished request (rs_server_release)."""
        self._keep.pop(ticket, None)
        return rs_server_release(self.handle, ticket)

    def stats(self):
        return rs_server_get_stats(self.handle)

    def close(self, cancel_pending: bool = False) -> None:
        if self.handle:
            rs_server_destroy(self.handle, cancel_pending)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan:
    """A sort captured into a CUDA graph (rs_plan_*).  algo: RS_PLAN_RADIX,
    RS_PLAN_BUCKET or RS_PLAN_SEGMENTED.  The tensors are kept referenced for
    the life of the plan; the constructor runs the sort (several times when
    autotuning) and waits for it."""

    def __init__(self, algo, keys_in, keys_out, vals_in=None, vals_out=None, key_bits: int = 0, min_key: int = 1,
                 max_key: int = 0, num_buckets: int = 0, seg_offsets=None, autotune: bool = False, ws=None):
        kb = key_bytes_of(keys_in)
        n = keys_in.numel()
        has_v = vals_in is not None
        nseg = seg_offsets.numel() - 1 if seg_offsets is not None else 0
        if ws is None:
            in_place = keys_out.data_ptr() == keys_in.data_ptr()
            if algo == RS_PLAN_SEGMENTED:
                nbytes = rs_segmented_workspace_bytes(kb, has_v, n, max(nseg, 1), key_bits)
            elif algo == RS_PLAN_BUCKET:
                nbytes = rs_workspace_bytes(RS_ALGO_BUCKET, kb, has_v, n, 0, num_buckets, in_place)
            else:
                nbytes = rs_workspace_bytes(RS_ALGO_RADIX, kb, has_v, n, key_bits, 0, in_place)
                if autotune:  # room for the shapes with wider digits too
                    for i in range(rs_config_count(kb, has_v)):
                        nbytes = max(nbytes, rs_workspace_bytes_cfg(kb, has_v, n, key_bits, rs_config_get(kb, has_v, i)))
            ws = workspace(nbytes, keys_in.device)
        self._keep = (keys_in, keys_out, vals_in, vals_out, seg_offsets, ws)
        desc = RsPlanDesc(algo, kb, keys_in.data_ptr(), keys_out.data_ptr(),
                          vals_in.data_ptr() if has_v else None, vals_out.data_ptr() if has_v else None, n, key_bits,
                          min_key, max_key, num_buckets, seg_offsets.data_ptr() if seg_offsets is not None else None,
                          nseg, ws.data_ptr(), ws.numel(), int(bool(autotune)))
        rc, self.handle = rs_plan_create(desc)
        check(rc, "rs_plan_create")
        self.ws = ws

    def launch(self, stream=None) -> None:
        check(rs_plan_launch(self.handle, stream), "rs_plan_launch")

    def info(self):
        rc, cfg, nodes, ms = rs_plan_info(self.handle)
        check(rc, "rs_plan_info")
        return cfg.as_tuple(), nodes, ms

    def close(self) -> None:
        if self.handle:
            rs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
