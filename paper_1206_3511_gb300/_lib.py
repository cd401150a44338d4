"""ctypes binding of librsort.so: one Python function per C entry point of
include/rsort.h, with the same name and argument order.  Arguments may be
torch tensors (their data pointer is passed), plain integers (raw device
addresses) or None (NULL).  A ``stream`` of None means torch's current stream
on the current device.  Nothing here computes; every step runs in the CUDA
library, and importing fails loudly if that library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsort.so")

_lock = threading.Lock()
_lib = None

_c = ctypes
_P = _c.c_void_p
_SZ = _c.c_size_t
_I = _c.c_int
_U32 = _c.c_uint32
_U64 = _c.c_uint64


class RsConfig(_c.Structure):
    _fields_ = [("digit_bits", _c.c_int), ("block_threads", _c.c_int), ("items_per_thread", _c.c_int)]

    def as_tuple(self):
        return (self.digit_bits, self.block_threads, self.items_per_thread)


class RsKernelStat(_c.Structure):
    _fields_ = [("name", _c.c_char * 32), ("launches", _c.c_uint64), ("total_ms", _c.c_double)]


class RsServerConfig(_c.Structure):
    _fields_ = [("pool", _c.c_void_p), ("pool_bytes", _c.c_size_t), ("budget_bytes", _c.c_size_t),
                ("num_streams", _c.c_int), ("max_batch", _c.c_int), ("batch_max_keys", _c.c_size_t)]


class RsRequest(_c.Structure):
    _fields_ = [("algo", _c.c_int), ("key_bytes", _c.c_int), ("keys_in", _c.c_void_p), ("keys_out", _c.c_void_p),
                ("vals_in", _c.c_void_p), ("vals_out", _c.c_void_p), ("n", _c.c_size_t), ("key_bits", _c.c_int),
                ("min_key", _c.c_uint64), ("max_key", _c.c_uint64), ("num_buckets", _c.c_size_t)]


class RsResult(_c.Structure):
    _fields_ = [("status", _c.c_int), ("t_arrive_ms", _c.c_double), ("t_start_ms", _c.c_double),
                ("t_done_ms", _c.c_double)]


class RsServerStats(_c.Structure):
    _fields_ = [("submitted", _c.c_uint64), ("completed", _c.c_uint64), ("rejected", _c.c_uint64),
                ("queued", _c.c_uint64), ("in_use_bytes", _c.c_size_t), ("max_in_use_bytes", _c.c_size_t),
                ("budget_bytes", _c.c_size_t), ("batches", _c.c_uint64), ("batched_requests", _c.c_uint64),
                ("max_queued", _c.c_uint64)]


class RsPlanDesc(_c.Structure):
    _fields_ = [("algo", _c.c_int), ("key_bytes", _c.c_int), ("keys_in", _c.c_void_p), ("keys_out", _c.c_void_p),
                ("vals_in", _c.c_void_p), ("vals_out", _c.c_void_p), ("n", _c.c_size_t), ("key_bits", _c.c_int),
                ("min_key", _c.c_uint64), ("max_key", _c.c_uint64), ("num_buckets", _c.c_size_t),
                ("d_seg_offsets", _c.c_void_p), ("nseg", _c.c_size_t), ("ws", _c.c_void_p),
                ("ws_bytes", _c.c_size_t), ("autotune", _c.c_int)]


# name -> (restype, argtypes)
SIGNATURES: dict[str, tuple] = {
    "rs_status_string": (_c.c_char_p, [_I]),
    "rs_version": (_I, []),
    "rs_default_config": (_I, [_I, _I, _SZ, _c.POINTER(RsConfig)]),
    "rs_config_count": (_I, [_I, _I]),
    "rs_config_get": (_I, [_I, _I, _I, _c.POINTER(RsConfig)]),
    "rs_workspace_bytes": (_SZ, [_I, _I, _I, _SZ, _I, _SZ, _I]),
    "rs_workspace_bytes_cfg": (_SZ, [_I, _I, _SZ, _I, _c.POINTER(RsConfig)]),
    "rs_sort_u32": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P]),
    "rs_sort_u64": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P]),
    "rs_sort_u32_ex": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "rs_sort_u64_ex": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "bs_sort_u32": (_I, [_P, _P, _P, _P, _SZ, _U32, _U32, _SZ, _P, _SZ, _P]),
    "bs_sort_u64": (_I, [_P, _P, _P, _P, _SZ, _U64, _U64, _SZ, _P, _SZ, _P]),
    "rs_digit_counts_u32": (_I, [_P, _SZ, _I, _I, _P, _P, _SZ, _P]),
    "rs_digit_counts_u64": (_I, [_P, _SZ, _I, _I, _P, _P, _SZ, _P]),
    "rs_counting_pass_u32": (_I, [_P, _P, _P, _P, _SZ, _I, _I, _P, _SZ, _P]),
    "rs_counting_pass_u64": (_I, [_P, _P, _P, _P, _SZ, _I, _I, _P, _SZ, _P]),
    "rs_segmented_workspace_bytes": (_SZ, [_I, _I, _SZ, _SZ, _I]),
    "rs_sort_segmented_u32": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P]),
    "rs_sort_segmented_u64": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P]),
    "rs_sort_segmented_u32_ex": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "rs_sort_segmented_u64_ex": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "bs_segmented_workspace_bytes": (_SZ, [_I, _I, _SZ, _SZ, _SZ]),
    "bs_sort_segmented_u32": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _U32, _U32, _SZ, _P, _SZ, _P]),
    "bs_sort_segmented_u64": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _U64, _U64, _SZ, _P, _SZ, _P]),
    "rs_sort_typed": (_I, [_I, _I, _I, _P, _P, _P, _P, _SZ, _P, _SZ, _P]),
    "bs_bucket_counts_u32": (_I, [_P, _SZ, _c.c_uint32, _c.c_uint32, _SZ, _P, _P, _SZ, _P]),
    "bs_bucket_counts_u64": (_I, [_P, _SZ, _c.c_uint64, _c.c_uint64, _SZ, _P, _P, _SZ, _P]),
    "rs_plan_create": (_I, [_c.POINTER(RsPlanDesc), _c.POINTER(_c.c_void_p)]),
    "rs_plan_launch": (_I, [_P, _P]),
    "rs_plan_info": (_I, [_P, _c.POINTER(RsConfig), _c.POINTER(_c.c_size_t), _c.POINTER(_c.c_float)]),
    "rs_plan_destroy": (None, [_P]),
    "rs_server_create": (_I, [_c.POINTER(RsServerConfig), _c.POINTER(_c.c_void_p)]),
    "rs_server_submit": (_I, [_P, _c.POINTER(RsRequest), _c.POINTER(_c.c_uint64)]),
    "rs_server_poll": (_I, [_P, _c.c_uint64, _c.POINTER(RsResult)]),
    "rs_server_wait": (_I, [_P, _c.c_uint64, _I]),
    "rs_server_release": (_I, [_P, _c.c_uint64]),
    "rs_server_get_stats": (_I, [_P, _c.POINTER(RsServerStats)]),
    "rs_server_destroy": (_I, [_P, _I]),
    "rs_sort_u32_noalloc": (_I, [_P, _P, _P, _P, _SZ, _I, _P]),
    "rs_host_sort_bytes": (_SZ, [_I, _I, _I, _SZ, _I, _SZ]),
    "rs_sort_host_u32": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P]),
    "rs_sort_host_u64": (_I, [_P, _P, _P, _P, _SZ, _I, _P, _SZ, _P]),
    "bs_sort_host_u32": (_I, [_P, _P, _P, _P, _SZ, _U32, _U32, _SZ, _P, _SZ, _P]),
    "bs_sort_host_u64": (_I, [_P, _P, _P, _P, _SZ, _U64, _U64, _SZ, _P, _SZ, _P]),
    "rs_segmented_host_bytes": (_SZ, [_I, _I, _SZ, _SZ, _I]),
    "rs_sort_segmented_host_u32": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "rs_sort_segmented_host_u64": (_I, [_P, _P, _P, _P, _P, _SZ, _SZ, _I, _P, _SZ, _P, _c.POINTER(RsConfig)]),
    "rs_get_status": (_I, [_P, _P]),
    "rs_set_debug": (None, [_U32, _I]),
    "rs_profile_enable": (None, [_I]),
    "rs_profile_read": (_I, [_c.POINTER(RsKernelStat), _I]),
    "rs_launch_count": (_U64, []),
    "rs_tune_cache_load": (_I, [_c.c_char_p]),
    "rs_tune_cache_save": (_I, [_c.c_char_p]),
    "rs_tune_cache_size": (_I, []),
    "rs_tune_cache_clear": (None, []),
}

STATUS = {
    0: "RS_OK", 1: "RS_ERR_INVALID_ARG", 2: "RS_ERR_WORKSPACE", 3: "RS_ERR_KEY_RANGE", 4: "RS_ERR_BUDGET",
    5: "RS_ERR_CUDA", 6: "RS_ERR_DEVICE_TIMEOUT", 7: "RS_ERR_NOT_READY", 8: "RS_ERR_SHUTDOWN",
    9: "RS_ERR_UNSUPPORTED",
    10: "RS_ERR_CHECK_FAILED",
}
RS_ALGO_RADIX = 0
RS_ALGO_BUCKET = 1


def load(path: str | None = None):
    """Load librsort.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(
                f"{p} is missing: the CUDA library has not been built "
                "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        lib = _c.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def ptr(x) -> int | None:
    """Device address of a tensor, an int address, or None for NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _call(name, *args):
    return getattr(load(), name)(*args)


# ---- one thin function per C entry point (same names, same argument order)
def rs_status_string(s: int) -> str:
    return _call("rs_status_string", s).decode()


def rs_version() -> int:
    return _call("rs_version")


def rs_default_config(key_bytes, has_values, n) -> RsConfig:
    cfg = RsConfig()
    rc = _call("rs_default_config", key_bytes, int(bool(has_values)), n, _c.byref(cfg))
    if rc:
        raise ValueError(STATUS.get(rc, rc))
    return cfg


def rs_config_count(key_bytes, has_values) -> int:
    return _call("rs_config_count", key_bytes, int(bool(has_values)))


def rs_config_get(key_bytes, has_values, i) -> RsConfig:
    cfg = RsConfig()
    rc = _call("rs_config_get", key_bytes, int(bool(has_values)), i, _c.byref(cfg))
    if rc:
        raise ValueError(STATUS.get(rc, rc))
    return cfg


def rs_workspace_bytes(algo, key_bytes, has_values, n, key_bits, num_buckets, in_place) -> int:
    return _call("rs_workspace_bytes", algo, key_bytes, int(bool(has_values)), n, key_bits, num_buckets,
                 int(bool(in_place)))


def rs_workspace_bytes_cfg(key_bytes, has_values, n, key_bits, cfg) -> int:
    return _call("rs_workspace_bytes_cfg", key_bytes, int(bool(has_values)), n, key_bits,
                 _c.byref(_as_cfg(cfg)))


def _as_cfg(cfg):
    if cfg is None or isinstance(cfg, RsConfig):
        return cfg
    return RsConfig(*cfg)


def rs_sort_u32(keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream=None) -> int:
    return _call("rs_sort_u32", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, key_bits, ptr(ws),
                 ws_bytes, stream_handle(stream))


def rs_sort_u64(keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream=None) -> int:
    return _call("rs_sort_u64", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, key_bits, ptr(ws),
                 ws_bytes, stream_handle(stream))


def rs_sort_u32_ex(keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_u32_ex", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, key_bits, ptr(ws),
                 ws_bytes, stream_handle(stream), _c.byref(c) if c is not None else None)


def rs_sort_u64_ex(keys_in, keys_out, vals_in, vals_out, n, key_bits, ws, ws_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_u64_ex", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, key_bits, ptr(ws),
                 ws_bytes, stream_handle(stream), _c.byref(c) if c is not None else None)


def bs_sort_u32(keys_in, keys_out, vals_in, vals_out, n, min_key, max_key, num_buckets, ws, ws_bytes,
                stream=None) -> int:
    return _call("bs_sort_u32", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, min_key, max_key,
                 num_buckets, ptr(ws), ws_bytes, stream_handle(stream))


def bs_sort_u64(keys_in, keys_out, vals_in, vals_out, n, min_key, max_key, num_buckets, ws, ws_bytes,
                stream=None) -> int:
    return _call("bs_sort_u64", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, min_key, max_key,
                 num_buckets, ptr(ws), ws_bytes, stream_handle(stream))


def rs_digit_counts_u32(keys, n, key_bits, digit_bits, counts_out, ws, ws_bytes, stream=None) -> int:
    return _call("rs_digit_counts_u32", ptr(keys), n, key_bits, digit_bits, ptr(counts_out), ptr(ws), ws_bytes,
                 stream_handle(stream))


def rs_digit_counts_u64(keys, n, key_bits, digit_bits, counts_out, ws, ws_bytes, stream=None) -> int:
    return _call("rs_digit_counts_u64", ptr(keys), n, key_bits, digit_bits, ptr(counts_out), ptr(ws), ws_bytes,
                 stream_handle(stream))


def rs_counting_pass_u32(keys_in, keys_out, vals_in, vals_out, n, shift, digit_bits, ws, ws_bytes,
                         stream=None) -> int:
    return _call("rs_counting_pass_u32", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, shift,
                 digit_bits, ptr(ws), ws_bytes, stream_handle(stream))


def rs_counting_pass_u64(keys_in, keys_out, vals_in, vals_out, n, shift, digit_bits, ws, ws_bytes,
                         stream=None) -> int:
    return _call("rs_counting_pass_u64", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, shift,
                 digit_bits, ptr(ws), ws_bytes, stream_handle(stream))


def rs_segmented_workspace_bytes(key_bytes, has_values, n_total, nseg, key_bits) -> int:
    return _call("rs_segmented_workspace_bytes", key_bytes, int(bool(has_values)), n_total, nseg, key_bits)


def rs_sort_segmented_u32(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws, ws_bytes,
                          stream=None) -> int:
    return _call("rs_sort_segmented_u32", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, key_bits, ptr(ws), ws_bytes, stream_handle(stream))


def rs_sort_segmented_u64(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws, ws_bytes,
                          stream=None) -> int:
    return _call("rs_sort_segmented_u64", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, key_bits, ptr(ws), ws_bytes, stream_handle(stream))


def bs_segmented_workspace_bytes(key_bytes, has_values, n_total, nseg, keys_per_bucket) -> int:
    return _call("bs_segmented_workspace_bytes", key_bytes, int(bool(has_values)), n_total, nseg, keys_per_bucket)


def bs_sort_segmented_u32(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, min_key, max_key,
                          keys_per_bucket, ws, ws_bytes, stream=None) -> int:
    return _call("bs_sort_segmented_u32", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, min_key, max_key, keys_per_bucket, ptr(ws), ws_bytes,
                 stream_handle(stream))


def bs_sort_segmented_u64(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, min_key, max_key,
                          keys_per_bucket, ws, ws_bytes, stream=None) -> int:
    return _call("bs_sort_segmented_u64", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, min_key, max_key, keys_per_bucket, ptr(ws), ws_bytes,
                 stream_handle(stream))


def rs_sort_segmented_u32_ex(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                             ws_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_segmented_u32_ex", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, key_bits, ptr(ws), ws_bytes, stream_handle(stream),
                 _c.byref(c) if c is not None else None)


def rs_sort_segmented_u64_ex(keys_in, keys_out, vals_in, vals_out, d_seg_offsets, nseg, n_total, key_bits, ws,
                             ws_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_segmented_u64_ex", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out),
                 ptr(d_seg_offsets), nseg, n_total, key_bits, ptr(ws), ws_bytes, stream_handle(stream),
                 _c.byref(c) if c is not None else None)


def bs_bucket_counts_u32(keys, n, min_key, max_key, num_buckets, d_counts, ws, ws_bytes, stream=None) -> int:
    return _call("bs_bucket_counts_u32", ptr(keys), n, min_key, max_key, num_buckets, ptr(d_counts), ptr(ws), ws_bytes,
                 stream_handle(stream))


def bs_bucket_counts_u64(keys, n, min_key, max_key, num_buckets, d_counts, ws, ws_bytes, stream=None) -> int:
    return _call("bs_bucket_counts_u64", ptr(keys), n, min_key, max_key, num_buckets, ptr(d_counts), ptr(ws), ws_bytes,
                 stream_handle(stream))


RS_KEY_UINT, RS_KEY_INT, RS_KEY_FLOAT = 0, 1, 2


def rs_sort_typed(key_kind, key_bytes, descending, keys_in, keys_out, vals_in, vals_out, n, ws, ws_bytes,
                  stream=None) -> int:
    return _call("rs_sort_typed", key_kind, key_bytes, int(bool(descending)), ptr(keys_in), ptr(keys_out),
                 ptr(vals_in), ptr(vals_out), n, ptr(ws), ws_bytes, stream_handle(stream))


RS_PLAN_RADIX, RS_PLAN_BUCKET, RS_PLAN_SEGMENTED = 0, 1, 2


def rs_plan_create(desc: RsPlanDesc):
    """Returns (status, plan handle)."""
    h = _c.c_void_p()
    rc = _call("rs_plan_create", _c.byref(desc), _c.byref(h))
    return rc, h.value


def rs_plan_launch(plan, stream=None) -> int:
    return _call("rs_plan_launch", plan, stream_handle(stream))


def rs_plan_info(plan):
    """Returns (status, RsConfig, kernel nodes, tuned ms)."""
    cfg = RsConfig()
    nodes = _c.c_size_t()
    ms = _c.c_float()
    rc = _call("rs_plan_info", plan, _c.byref(cfg), _c.byref(nodes), _c.byref(ms))
    return rc, cfg, nodes.value, ms.value


def rs_plan_destroy(plan) -> None:
    _call("rs_plan_destroy", plan)


def rs_server_create(cfg: RsServerConfig):
    """Returns (status, server handle)."""
    h = _c.c_void_p()
    rc = _call("rs_server_create", _c.byref(cfg), _c.byref(h))
    return rc, h.value


def rs_server_submit(server, req: RsRequest):
    """Returns (status, ticket)."""
    t = _c.c_uint64()
    rc = _call("rs_server_submit", server, _c.byref(req), _c.byref(t))
    return rc, t.value


def rs_server_poll(server, ticket):
    """Returns (status, RsResult)."""
    r = RsResult()
    rc = _call("rs_server_poll", server, ticket, _c.byref(r))
    return rc, r


def rs_server_release(server, ticket) -> int:
    return _call("rs_server_release", server, ticket)


def rs_server_wait(server, ticket, timeout_ms=-1) -> int:
    return _call("rs_server_wait", server, ticket, timeout_ms)


def rs_server_get_stats(server) -> RsServerStats:
    st = RsServerStats()
    rc = _call("rs_server_get_stats", server, _c.byref(st))
    if rc:
        raise RuntimeError(STATUS.get(rc, rc))
    return st


def rs_server_destroy(server, cancel_pending=False) -> int:
    return _call("rs_server_destroy", server, int(bool(cancel_pending)))


RS_NOALLOC_MAX_KEYS = 1 << 20


def rs_sort_u32_noalloc(keys_in, keys_out, vals_in, vals_out, n, key_bits, stream=None) -> int:
    """rs_sort_u32 for callers that cannot allocate: the scratch is a fixed
    array inside the library (n <= RS_NOALLOC_MAX_KEYS; calls must not
    overlap on the GPU)."""
    return _call("rs_sort_u32_noalloc", ptr(keys_in), ptr(keys_out), ptr(vals_in), ptr(vals_out), n, key_bits,
                 stream_handle(stream))


def rs_host_sort_bytes(algo, key_bytes, has_values, n, key_bits, num_buckets) -> int:
    return _call("rs_host_sort_bytes", algo, key_bytes, int(bool(has_values)), n, key_bits, num_buckets)


def rs_sort_host_u32(h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, key_bits, dev_buf, dev_buf_bytes,
                     stream=None) -> int:
    """Host pointers in and out; dev_buf is a device buffer of
    rs_host_sort_bytes(...) bytes."""
    return _call("rs_sort_host_u32", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out), n, key_bits,
                 ptr(dev_buf), dev_buf_bytes, stream_handle(stream))


def rs_sort_host_u64(h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, key_bits, dev_buf, dev_buf_bytes,
                     stream=None) -> int:
    return _call("rs_sort_host_u64", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out), n, key_bits,
                 ptr(dev_buf), dev_buf_bytes, stream_handle(stream))


def bs_sort_host_u32(h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, min_key, max_key, num_buckets, dev_buf,
                     dev_buf_bytes, stream=None) -> int:
    return _call("bs_sort_host_u32", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out), n, min_key,
                 max_key, num_buckets, ptr(dev_buf), dev_buf_bytes, stream_handle(stream))


def bs_sort_host_u64(h_keys_in, h_keys_out, h_vals_in, h_vals_out, n, min_key, max_key, num_buckets, dev_buf,
                     dev_buf_bytes, stream=None) -> int:
    return _call("bs_sort_host_u64", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out), n, min_key,
                 max_key, num_buckets, ptr(dev_buf), dev_buf_bytes, stream_handle(stream))


def rs_segmented_host_bytes(key_bytes, has_values, n_total, nseg, key_bits) -> int:
    return _call("rs_segmented_host_bytes", key_bytes, int(bool(has_values)), n_total, nseg, key_bits)


def rs_sort_segmented_host_u32(h_keys_in, h_keys_out, h_vals_in, h_vals_out, h_seg_offsets, nseg, n_total, key_bits,
                               dev_buf, dev_buf_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_segmented_host_u32", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out),
                 ptr(h_seg_offsets), nseg, n_total, key_bits, ptr(dev_buf), dev_buf_bytes, stream_handle(stream),
                 _c.byref(c) if c is not None else None)


def rs_sort_segmented_host_u64(h_keys_in, h_keys_out, h_vals_in, h_vals_out, h_seg_offsets, nseg, n_total, key_bits,
                               dev_buf, dev_buf_bytes, stream=None, cfg=None) -> int:
    c = _as_cfg(cfg)
    return _call("rs_sort_segmented_host_u64", ptr(h_keys_in), ptr(h_keys_out), ptr(h_vals_in), ptr(h_vals_out),
                 ptr(h_seg_offsets), nseg, n_total, key_bits, ptr(dev_buf), dev_buf_bytes, stream_handle(stream),
                 _c.byref(c) if c is not None else None)


def rs_tune_cache_load(path: str) -> int:
    return _call("rs_tune_cache_load", os.fsencode(path))


def rs_tune_cache_save(path: str) -> int:
    return _call("rs_tune_cache_save", os.fsencode(path))


def rs_tune_cache_size() -> int:
    return _call("rs_tune_cache_size")


def rs_tune_cache_clear() -> None:
    _call("rs_tune_cache_clear")


def rs_get_status(ws, stream=None) -> int:
    return _call("rs_get_status", ptr(ws), stream_handle(stream))


def rs_set_debug(spin_limit: int, stall_tile: int) -> None:
    _call("rs_set_debug", spin_limit, stall_tile)


def rs_profile_enable(enable: bool) -> None:
    _call("rs_profile_enable", int(bool(enable)))


def rs_profile_read(cap: int = 32) -> dict[str, tuple[int, float]]:
    """{kernel name: (launches, total ms)} of the events recorded since the
    last read (waits for them)."""
    arr = (RsKernelStat * cap)()
    k = _call("rs_profile_read", arr, cap)
    if k < 0:
        raise RuntimeError("rs_profile_read: CUDA error while reading events")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(k)}


def rs_launch_count() -> int:
    return int(_call("rs_launch_count"))
