"""GPU parity of the host-buffer sorts (rs_sort_host_*, bs_sort_host_*):
keys and values in host memory, copied in, sorted on the device and copied
back by one call; the result must equal the oracle bit for bit."""
import numpy as np
import pytest

import synth
from tests._util import assert_same

pytestmark = pytest.mark.gpu


def _host(a: np.ndarray, pinned: bool):
    import torch

    signed = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}[a.dtype]
    t = torch.from_numpy(np.ascontiguousarray(a).view(signed)).clone()
    return t.pin_memory() if pinned else t


def _np(t, dtype):
    return t.numpy().view(dtype)


@pytest.mark.parametrize("kb,with_values,key_bits,pinned,n", [
    (4, False, 0, True, 1_000_003),
    (4, True, 0, False, 300_001),
    (8, False, 40, True, 777_777),
    (8, True, 0, True, 250_000),
    (4, False, 0, True, 3000),      # one block sorts it in shared memory
])
def test_radix_host_sort_matches_oracle(rs, oracle, kb, with_values, key_bits, pinned, n):
    import torch

    keys = synth.u32(n, 501, 0) if kb == 4 else synth.keys_u64(n, key_bits or 64, seed=502)
    vals = synth.index_values(n) if with_values else None
    hk = _host(keys, pinned)
    hv = _host(vals, pinned) if with_values else None
    stream = torch.cuda.Stream()
    ok, ov = rs.sort_host(hk, hv, key_bits=key_bits, stream=stream)
    stream.synchronize()
    kbits = key_bits or 8 * kb
    if with_values:
        wk, wv = oracle.radix_sort(keys, vals, kbits)
        assert_same(_np(ov, np.uint32), wv, "host radix values")
    else:
        wk = oracle.radix_sort(keys, None, kbits)
    assert_same(_np(ok, keys.dtype), wk, "host radix keys")
    assert_same(_np(hk, keys.dtype), keys, "input left unchanged")


def test_radix_host_sort_in_place_and_status(rs, oracle):
    import torch

    n = 2_000_000
    keys = synth.keys_u32(n, 6, seed=503)
    hk = _host(keys, True)
    nbytes = rs.rs_host_sort_bytes(rs.RS_ALGO_RADIX, 4, 0, n, 0, 0)
    buf = rs.workspace(nbytes)
    stream = torch.cuda.Stream()
    assert rs.rs_sort_host_u32(hk, hk, None, None, n, 0, buf, nbytes, stream) == 0
    assert rs.rs_get_status(buf, stream) == 0
    assert_same(_np(hk, np.uint32), oracle.radix_sort(keys, None, 32), "in place")


@pytest.mark.parametrize("kb,with_values,bounds", [(4, False, False), (4, True, True), (8, True, False)])
def test_bucket_host_sort_matches_oracle(rs, oracle, kb, with_values, bounds):
    import torch

    n = 600_001
    keys = synth.keys_u32(n, 0, seed=504) if kb == 4 else synth.keys_u64(n, 48, seed=505)
    vals = synth.index_values(n) if with_values else None
    lo, hi = int(keys.min()), int(keys.max())
    hk = _host(keys, True)
    hv = _host(vals, True) if with_values else None
    stream = torch.cuda.Stream()
    kw = dict(min_key=lo, max_key=hi) if bounds else {}
    ok, ov = rs.sort_host(hk, hv, algo=rs.RS_ALGO_BUCKET, num_buckets=n // 16, stream=stream, **kw)
    stream.synchronize()
    if with_values:
        wk, wv = oracle.bucket_sort(keys, vals, lo, hi, n // 16)
        assert_same(_np(ov, np.uint32), wv, "host bucket values")
    else:
        wk = oracle.bucket_sort(keys, None, lo, hi, n // 16)
    assert_same(_np(ok, keys.dtype), wk, "host bucket keys")


def test_host_sorts_on_two_streams_overlap_and_stay_correct(rs, oracle):
    """Two calls on two streams with their own device buffers: both correct."""
    import torch

    n = 4_000_000
    a = synth.u32(n, 506, 0)
    b = synth.keys_u32(n, 4, seed=507)
    ha, hb = _host(a, True), _host(b, True)
    oa, ob = torch.empty_like(ha).pin_memory(), torch.empty_like(hb).pin_memory()
    nbytes = rs.rs_host_sort_bytes(rs.RS_ALGO_RADIX, 4, 0, n, 0, 0)
    bufs = [rs.workspace(nbytes), rs.workspace(nbytes)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for _ in range(2):
        assert rs.rs_sort_host_u32(ha, oa, None, None, n, 0, bufs[0], nbytes, streams[0]) == 0
        assert rs.rs_sort_host_u32(hb, ob, None, None, n, 0, bufs[1], nbytes, streams[1]) == 0
    torch.cuda.synchronize()
    assert_same(_np(oa, np.uint32), np.sort(a), "stream 0")
    assert_same(_np(ob, np.uint32), np.sort(b), "stream 1")


def test_host_sort_rejects_device_arrays_and_small_buffers(rs):
    import torch

    n = 10_000
    hk = torch.zeros(n, dtype=torch.int32).pin_memory()
    dk = torch.zeros(n, dtype=torch.int32, device="cuda")
    nbytes = rs.rs_host_sort_bytes(rs.RS_ALGO_RADIX, 4, 0, n, 0, 0)
    buf = rs.workspace(nbytes)
    # device memory where host arrays belong
    assert rs.rs_sort_host_u32(dk, hk, None, None, n, 0, buf, nbytes, None) == 1
    # host memory as the device buffer, and a buffer too small
    assert rs.rs_sort_host_u32(hk, hk, None, None, n, 0, hk, nbytes, None) == 2
    assert rs.rs_sort_host_u32(hk, hk, None, None, n, 0, buf, nbytes - 256, None) == 2
    torch.cuda.synchronize()


@pytest.mark.parametrize("kb,with_values", [(4, False), (8, True)])
def test_segmented_host_sort_matches_oracle(rs, oracle, kb, with_values):
    import torch

    sizes = synth.log_uniform_sizes(300, 1, 60_000, seed=508)
    n = int(sizes.sum())
    off = synth.segment_offsets(sizes).astype(np.uint64)
    keys = synth.u32(n, 509, 0) if kb == 4 else synth.keys_u64(n, 64, seed=509)
    vals = synth.index_values(n) if with_values else None
    hk = _host(keys, True)
    hv = _host(vals, True) if with_values else None
    ok = torch.empty_like(hk).pin_memory()
    ov = torch.empty_like(hv).pin_memory() if with_values else None
    ho = _host(off, True)
    nbytes = rs.rs_segmented_host_bytes(kb, with_values, n, len(sizes), 0)
    buf = rs.workspace(nbytes)
    stream = torch.cuda.Stream()
    fn = rs.rs_sort_segmented_host_u32 if kb == 4 else rs.rs_sort_segmented_host_u64
    assert fn(hk, ok, hv, ov, ho, len(sizes), n, 0, buf, nbytes, stream) == 0
    assert rs.rs_get_status(buf, stream) == 0
    if with_values:
        wk, wv = oracle.segmented_radix_sort(keys, off, vals, 8 * kb)
        assert_same(_np(ov, np.uint32), wv, "segmented host values")
    else:
        wk = oracle.segmented_radix_sort(keys, off, None, 8 * kb)
    assert_same(_np(ok, keys.dtype), wk, "segmented host keys")
