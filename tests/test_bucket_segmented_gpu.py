"""GPU parity of the segmented bucket sort (bs_sort_segmented_u32/u64): every
segment must equal the oracle's bucket sort of that segment alone
(Algorithm 2 with Algorithm 1 per bucket, the segment's own bounds and
max(1, n // keys_per_bucket) buckets), keys and values, zero tolerance."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _run(rs, keys, sizes, vals=None, lo=None, hi=None, kpb=0, in_place=False):
    import torch

    off = synth.segment_offsets(sizes)
    kd = to_dev(keys)
    vd = to_dev(vals) if vals is not None else None
    od = to_dev(off.astype(np.uint64))
    if in_place:
        ok, ov = rs.segmented_bucket_sort(kd, od, vd, lo, hi, kpb, out=kd, out_values=vd)
    else:
        ok, ov = rs.segmented_bucket_sort(kd, od, vd, lo, hi, kpb)
    torch.cuda.synchronize()
    return off, from_dev(ok, keys.dtype), (from_dev(ov, np.uint32) if vals is not None else None)


def _check(rs, oracle, keys, sizes, vals=None, lo=None, hi=None, kpb=0, in_place=False, what="",
           bucket_oracle=True):
    off, gk, gv = _run(rs, keys, sizes, vals, lo, hi, kpb, in_place)
    per = kpb or 16
    for s in range(len(sizes)):
        a, b = int(off[s]), int(off[s + 1])
        if a == b:
            continue
        sv = vals[a:b] if vals is not None else None
        if bucket_oracle:
            want = oracle.bucket_sort(keys[a:b], sv, lo, hi, max(1, (b - a) // per))
        else:
            want = oracle.radix_sort(keys[a:b], sv)
        if vals is None:
            assert_same(gk[a:b], want, f"{what} segment {s} (n={b - a})")
        else:
            assert_same(gk[a:b], want[0], f"{what} segment {s} (n={b - a}) keys")
            assert_same(gv[a:b], want[1], f"{what} segment {s} (n={b - a}) values")


def _sizes(count, lo, hi, seed):
    sizes = synth.log_uniform_sizes(count, lo, hi, seed=seed, dist_id=50).astype(np.int64)
    # empty, one-key and small/large boundary segments among them
    sizes[:8] = [0, 1, 2, 4096, 4097, 0, 16, 70_000]
    return sizes


@pytest.mark.parametrize("kb,with_values", [(4, False), (4, True), (8, False), (8, True)])
def test_log_uniform_segments_computed_bounds(rs, oracle, kb, with_values):
    """300 segments, sizes log-uniform in [1, 300000], each bucket-sorted over
    its own min and max."""
    sizes = _sizes(300, 1, 300_000, 7 + kb)
    n = int(sizes.sum())
    keys = synth.u32(n, 51, 0) if kb == 4 else synth.keys_u64(n, 64, seed=51)
    vals = synth.index_values(n) if with_values else None
    _check(rs, oracle, keys, sizes, vals, what=f"computed kb={kb} v={with_values}")


@pytest.mark.parametrize("dist", [0, 1, 3, 4, 5])
def test_declared_bounds_per_distribution(rs, oracle, dist):
    """Segments of one benchmark distribution with its declared bounds for
    every segment."""
    sizes = _sizes(120, 1, 200_000, 20 + dist)
    n = int(sizes.sum())
    keys = synth.keys_u32(n, dist, seed=dist)
    lo, hi = synth.DECLARED_BOUNDS[dist]
    _check(rs, oracle, keys, sizes, synth.index_values(n), lo, hi, what=synth.DISTS[dist])


def test_segments_whose_keys_are_all_equal(rs, oracle):
    """min == max in a segment: one possible key, nothing to sort (small and
    large segments), next to ordinary ones."""
    sizes = np.array([1, 3, 5000, 40_000, 300, 9000], np.int64)
    n = int(sizes.sum())
    keys = synth.u32(n, 52, 0)
    off = synth.segment_offsets(sizes)
    for s in (1, 3, 4):
        keys[int(off[s]):int(off[s + 1])] = 12345 + s
    _check(rs, oracle, keys, sizes, synth.index_values(n), what="constant segments")


@pytest.mark.parametrize("kpb", [1, 4, 64, 1000])
def test_keys_per_bucket(rs, oracle, kpb):
    """keys_per_bucket 1 is the paper's n buckets; larger values make fewer,
    fuller buckets (and, for large segments with few buckets, partitions that
    stay above the shared-memory size at level 2: the overflow radix)."""
    sizes = _sizes(80, 1, 150_000, 30 + kpb)
    n = int(sizes.sum())
    keys = synth.u32(n, 53, 0) >> np.uint32(4)
    _check(rs, oracle, keys, sizes, synth.index_values(n), kpb=kpb, what=f"kpb={kpb}")


def test_skewed_keys_take_the_overflow_path(rs, oracle):
    """Gaussian keys (sd 2^20) with the full 32-bit range declared: the keys
    crowd into a few dozen buckets of ~10,000 keys, which level 2 cannot
    split further; those partitions are radix-sorted on their key bits."""
    sizes = np.array([500_000, 3000, 800_000, 10], np.int64)
    n = int(sizes.sum())
    keys = synth.keys_u32(n, 6, seed=54)
    _check(rs, oracle, keys, sizes, synth.index_values(n), 0, 2**32 - 1, what="gaussian", bucket_oracle=False)
    keys64 = synth.keys_u64_shaped(n, 6, seed=55)
    _check(rs, oracle, keys64, sizes, synth.index_values(n), 0, 2**64 - 1, what="gaussian u64",
           bucket_oracle=False)


@pytest.mark.parametrize("kb", [4, 8])
def test_in_place(rs, oracle, kb):
    sizes = _sizes(60, 1, 100_000, 40 + kb)
    n = int(sizes.sum())
    keys = synth.u32(n, 56, 0) if kb == 4 else synth.keys_u64(n, 64, seed=56)
    _check(rs, oracle, keys, sizes, synth.index_values(n), in_place=True, what=f"in place kb={kb}")


@pytest.mark.parametrize("where", [100, 20_000])
def test_key_outside_declared_bounds_is_reported(rs, where):
    """A key above max_key in a small (shared-memory) or a large segment."""
    import torch

    sizes = [1000, 30_000, 500]
    n = sum(sizes)
    keys = synth.u32(n, 57, 0) >> np.uint32(12)  # 20-bit keys
    keys[where] = 1 << 20
    kd = to_dev(keys)
    od = to_dev(synth.segment_offsets(sizes).astype(np.uint64))
    ws = rs.workspace(rs.bs_segmented_workspace_bytes(4, 0, n, 3, 0))
    out = torch.empty_like(kd)
    assert rs.bs_sort_segmented_u32(kd, out, None, None, od, 3, n, 0, (1 << 20) - 1, 0, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE


def test_offsets_past_n_total_are_reported_and_nothing_is_written_outside(rs, oracle):
    import torch

    sizes = [3000, 70_000, 100]
    n = sum(sizes)
    keys = synth.u32(n, 58, 0)
    off = synth.segment_offsets(sizes).astype(np.uint64)
    off[-1] = n + 7
    G = 1 << 16
    guard = -0x21524111
    kd = to_dev(keys)
    out = torch.full((n + 2 * G,), guard, dtype=torch.int32, device="cuda")
    wsb = rs.bs_segmented_workspace_bytes(4, 0, n, 3, 0)
    wsbuf = torch.full((wsb + G,), 0x5A, dtype=torch.uint8, device="cuda")
    ws = wsbuf[:wsb]
    assert rs.bs_sort_segmented_u32(kd, out[G:G + n], None, None, to_dev(off), 3, n, 1, 0, 0, ws, wsb) == 0
    assert rs.get_status(ws) == 1  # RS_ERR_INVALID_ARG
    o = out.cpu().numpy()
    assert np.all(o[:G] == guard) and np.all(o[G + n:] == guard)
    assert np.all(wsbuf[wsb:].cpu().numpy() == 0x5A)
    got = o[G:G + n].view(np.uint32)
    for a, b in [(0, 3000), (3000, 73_000)]:
        assert_same(got[a:b], oracle.bucket_sort(keys[a:b]), f"segment [{a},{b})")


def test_argument_errors(rs):
    import torch

    kd = torch.zeros(10, dtype=torch.int32, device="cuda")
    od = to_dev(np.array([0, 10], np.uint64))
    ws = rs.workspace(rs.bs_segmented_workspace_bytes(4, 0, 10, 1, 0))
    v = torch.zeros(10, dtype=torch.int32, device="cuda")
    assert rs.bs_sort_segmented_u32(kd, kd, v, None, od, 1, 10, 1, 0, 0, ws, ws.numel()) == 1
    assert rs.bs_sort_segmented_u32(kd, kd, None, None, od, 1, 10, 1, 0, 0, None, 0) == 2
    assert rs.bs_sort_segmented_u32(kd, kd, None, None, od, 0, 0, 1, 0, 0, ws, ws.numel()) == 0  # no segments
