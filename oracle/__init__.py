"""CPU oracle for the bucket sort and LSD radix sort of Horsmalahti,
"Comparison of Bucket Sort and RADIX Sort" (arXiv:1206.3511).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports this package, and this package imports nothing from the library.

The arithmetic lives in ``oracle.c`` (plain C, one routine per step of the
paper's Algorithms 1-4).  This module compiles it with gcc on first use and
wraps it with ctypes.  32-bit keys are widened to 64 bits before the call and
narrowed after it; the C code only ever sees uint64 keys and uint32 values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P64 = ctypes.POINTER(ctypes.c_uint64)
            P32 = ctypes.POINTER(ctypes.c_uint32)
            sz, i = ctypes.c_size_t, ctypes.c_int
            u64 = ctypes.c_uint64
            lib.oracle_counting_pass_u64.argtypes = [P64, P32, P64, P32, sz, i, i]
            lib.oracle_counting_pass_backward_u64.argtypes = [P64, P32, P64, P32, sz, i, i]
            lib.oracle_num_passes.argtypes = [i, i]
            lib.oracle_digit_counts_u64.argtypes = [P64, sz, i, i, P64]
            lib.oracle_radix_sort_partial_u64.argtypes = [P64, P32, sz, i, i, i, P64, P32]
            lib.oracle_radix_sort_u64.argtypes = [P64, P32, sz, i, i, P64, P32]
            lib.oracle_bucket_index_u64.argtypes = [u64, u64, u64, u64]
            lib.oracle_bucket_index_u64.restype = u64
            lib.oracle_bucket_counts_u64.argtypes = [P64, sz, u64, u64, u64, P64]
            lib.oracle_bucket_sort_u64.argtypes = [P64, P32, sz, u64, u64, u64, P64, P32]
            lib.oracle_minmax_u64.argtypes = [P64, sz, P64, P64]
            lib.oracle_sort_typed_u64.argtypes = [P64, P32, sz, i, i, i, P64, P32]
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


_ERRORS = {-1: "bad argument", -2: "key outside the declared range", -3: "out of memory"}


def _check(rc: int) -> None:
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"oracle error {rc}"))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if a is not None else None


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if a is not None else None


def _widen(keys) -> tuple[np.ndarray, np.dtype]:
    keys = np.asarray(keys)
    if keys.dtype not in (np.uint32, np.uint64):
        raise TypeError(f"oracle keys must be uint32 or uint64, got {keys.dtype}")
    return np.ascontiguousarray(keys, dtype=np.uint64), keys.dtype


def _vals(vals, n):
    if vals is None:
        return None
    v = np.ascontiguousarray(vals, dtype=np.uint32)
    if v.shape != (n,):
        raise ValueError("values must have one entry per key")
    return v


def num_passes(key_bits: int, digit_bits: int) -> int:
    """ceil(key_bits / digit_bits): the d of Algorithm 4 for D-bit digits."""
    return _load().oracle_num_passes(key_bits, digit_bits)


def counting_pass(keys, vals=None, shift: int = 0, digit_bits: int = 8, backward: bool = False):
    """One stable counting sort (Algorithm 3) of the array on digit
    (k >> shift) & (2^digit_bits - 1).  ``backward=True`` runs the paper's
    printed form (inclusive prefix, backward placement)."""
    k64, dt = _widen(keys)
    n = k64.size
    v = _vals(vals, n)
    out = np.empty(n, np.uint64)
    outv = np.empty(n, np.uint32) if v is not None else None
    fn = _load().oracle_counting_pass_backward_u64 if backward else _load().oracle_counting_pass_u64
    _check(fn(_p64(k64), _p32(v), _p64(out), _p32(outv), n, shift, digit_bits))
    return (out.astype(dt), outv) if v is not None else out.astype(dt)


def digit_counts(keys, key_bits: int, digit_bits: int = 8) -> np.ndarray:
    """counts[p, d] = number of keys whose digit p equals d (Algorithm 3's
    counting loop, for every pass of Algorithm 4)."""
    k64, _ = _widen(keys)
    P = num_passes(key_bits, digit_bits)
    out = np.empty((P, 1 << digit_bits), np.uint64)
    _check(_load().oracle_digit_counts_u64(_p64(k64), k64.size, key_bits, digit_bits, _p64(out)))
    return out


def radix_sort(keys, vals=None, key_bits: int | None = None, digit_bits: int = 8, max_passes: int = -1):
    """LSD radix sort (Algorithm 4 over Algorithm 3).  ``key_bits`` defaults to
    the key width.  With ``max_passes`` >= 0, returns the array after that many
    digit passes."""
    k64, dt = _widen(keys)
    if key_bits is None:
        key_bits = 8 * dt.itemsize
    n = k64.size
    v = _vals(vals, n)
    out = np.empty(n, np.uint64)
    outv = np.empty(n, np.uint32) if v is not None else None
    _check(_load().oracle_radix_sort_partial_u64(_p64(k64), _p32(v), n, key_bits, digit_bits,
                                                  max_passes, _p64(out), _p32(outv)))
    return (out.astype(dt), outv) if v is not None else out.astype(dt)


def bucket_index(key: int, min_key: int, max_key: int, nb: int) -> int:
    """floor((key - min) * nb / (max - min + 1)), exact (reading of Sec. 2.3)."""
    return int(_load().oracle_bucket_index_u64(key, min_key, max_key, nb))


def bucket_counts(keys, min_key: int, max_key: int, nb: int) -> np.ndarray:
    """Sizes of the nb bucket lists after Algorithm 2's insert loop."""
    k64, _ = _widen(keys)
    out = np.empty(nb, np.uint64)
    _check(_load().oracle_bucket_counts_u64(_p64(k64), k64.size, min_key, max_key, nb, _p64(out)))
    return out


def bucket_sort(keys, vals=None, min_key: int | None = None, max_key: int | None = None,
                nb: int | None = None):
    """Bucket sort (Algorithm 2 with Algorithm 1 per bucket).  Bounds default
    to the keys' own min and max; nb defaults to max(1, n // 16)."""
    k64, dt = _widen(keys)
    n = k64.size
    v = _vals(vals, n)
    if min_key is None or max_key is None:
        if n == 0:
            min_key, max_key = 0, 0
        else:
            lo, hi = minmax(k64)
            min_key = lo if min_key is None else min_key
            max_key = hi if max_key is None else max_key
    if nb is None:
        nb = max(1, n // 16)
    out = np.empty(n, np.uint64)
    outv = np.empty(n, np.uint32) if v is not None else None
    _check(_load().oracle_bucket_sort_u64(_p64(k64), _p32(v), n, min_key, max_key, nb,
                                          _p64(out), _p32(outv)))
    return (out.astype(dt), outv) if v is not None else out.astype(dt)


def minmax(keys) -> tuple[int, int]:
    """Smallest and largest key."""
    k64, _ = _widen(keys)
    lo = np.zeros(1, np.uint64)
    hi = np.zeros(1, np.uint64)
    _check(_load().oracle_minmax_u64(_p64(k64), k64.size, _p64(lo), _p64(hi)))
    return int(lo[0]), int(hi[0])


def segmented_radix_sort(keys, offsets, vals=None, key_bits: int | None = None, digit_bits: int = 8):
    """Each segment [offsets[s], offsets[s+1]) sorted on its own with
    ``radix_sort``; the segmented GPU sort must match this segment by segment."""
    keys = np.asarray(keys)
    offsets = np.asarray(offsets, dtype=np.int64)
    out = np.empty_like(keys)
    outv = np.empty(keys.size, np.uint32) if vals is not None else None
    for s in range(offsets.size - 1):
        a, b = int(offsets[s]), int(offsets[s + 1])
        if b == a:
            continue
        if vals is not None:
            ok, ov = radix_sort(keys[a:b], np.asarray(vals)[a:b], key_bits, digit_bits)
            out[a:b], outv[a:b] = ok, ov
        else:
            out[a:b] = radix_sort(keys[a:b], None, key_bits, digit_bits)
    return (out, outv) if vals is not None else out


KIND_UINT, KIND_INT, KIND_FLOAT = 0, 1, 2
_KIND_OF = {np.dtype(np.uint32): 0, np.dtype(np.uint64): 0, np.dtype(np.int32): 1, np.dtype(np.int64): 1,
            np.dtype(np.float32): 2, np.dtype(np.float64): 2}
_BITS_OF = {4: np.uint32, 8: np.uint64}


def sort_typed(keys, vals=None, kind: int | None = None, descending: bool = False):
    """Stable sort of typed keys (unsigned, signed, IEEE float by totalOrder),
    ascending or descending.  keys: a numpy array of a 4- or 8-byte dtype;
    kind None takes it from the dtype.  Returns keys (same dtype) or
    (keys, values)."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype.itemsize not in (4, 8):
        raise TypeError("keys must be 4 or 8 bytes wide")
    if kind is None:
        kind = _KIND_OF[keys.dtype]
    bits = keys.view(_BITS_OF[keys.dtype.itemsize]).astype(np.uint64)
    v = _vals(vals, bits.size)
    out = np.empty(bits.size, np.uint64)
    vout = np.empty(bits.size, np.uint32) if v is not None else None
    _check(_load().oracle_sort_typed_u64(_p64(bits), _p32(v), bits.size, keys.dtype.itemsize, kind,
                                         int(bool(descending)), _p64(out), _p32(vout)))
    res = out.astype(_BITS_OF[keys.dtype.itemsize]).view(keys.dtype)
    return res if v is None else (res, vout)
