"""GPU parity of the bucket sort (Algorithm 2) against the CPU oracle's
bucket sort, element by element, zero tolerance.  The oracle's bucket sort is
pinned equal to its radix sort and to stable library sorts, so the GPU bucket
sort is also compared with the oracle radix sort at sizes where the oracle's
insertion sorts would take too long."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _bucket(rs, keys, vals=None, lo=None, hi=None, nb=0, in_place=False):
    import torch

    kd = to_dev(keys)
    vd = to_dev(vals) if vals is not None else None
    if in_place:
        ok, ov = rs.bucket_sort(kd, vd, lo, hi, nb, out=kd, out_values=vd)
    else:
        ok, ov = rs.bucket_sort(kd, vd, lo, hi, nb)
    torch.cuda.synchronize()
    return from_dev(ok, keys.dtype), (from_dev(ov, np.uint32) if vals is not None else None)


def _check(rs, oracle, keys, vals=None, lo=None, hi=None, nb=0, in_place=False, what="", use_bucket_oracle=True):
    gk, gv = _bucket(rs, keys, vals, lo, hi, nb, in_place)
    if use_bucket_oracle:
        want = oracle.bucket_sort(keys, vals, lo, hi, nb or max(1, keys.size // 16))
    else:
        want = oracle.radix_sort(keys, vals)
    if vals is None:
        assert_same(gk, want, what)
    else:
        assert_same(gk, want[0], what + " keys")
        assert_same(gv, want[1], what + " values")


def test_small_config_1m_uniform_31bit(rs, oracle):
    """1,000,000 u32 keys uniform in [0, 2^31), seed 0, 62,500 buckets over
    [0, 2^31 - 1]."""
    keys = synth.u32(1_000_000, 0, 0) >> np.uint32(1)
    _check(rs, oracle, keys, None, 0, 2**31 - 1, 62_500, what="1M uniform")


@pytest.mark.parametrize("dist", list(synth.DISTS))
def test_distributions_declared_bounds(rs, oracle, dist):
    n = 200_003
    keys = synth.keys_u32(n, dist, seed=3)
    lo, hi = synth.DECLARED_BOUNDS[dist]
    _check(rs, oracle, keys, synth.index_values(n), lo, hi, 0, what=synth.DISTS[dist],
           use_bucket_oracle=dist not in (6,))


@pytest.mark.parametrize("dist", [0, 1, 6, 8])
def test_distributions_computed_bounds(rs, oracle, dist):
    n = 150_001
    keys = synth.keys_u32(n, dist, seed=4)
    _check(rs, oracle, keys, synth.index_values(n), None, None, 0, what="computed " + synth.DISTS[dist],
           use_bucket_oracle=False)


@pytest.mark.parametrize("n", [1, 2, 3, 16, 17, 4095, 4096, 4097, 65_537, 1_048_577])
def test_sizes(rs, oracle, n):
    keys = synth.u32(n, 50, 0)
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**32 - 1, 0, what=f"n={n}", use_bucket_oracle=n < 100_000)


@pytest.mark.parametrize("nb", [1, 2, 3, 255, 256, 257, 4096, 65_536, 300_000, 2_000_000])
def test_bucket_counts(rs, oracle, nb):
    """nb = 1 (one bucket), nb around the level boundaries, nb > n and nb > range."""
    n = 300_000
    keys = synth.u32(n, 51, 0) >> np.uint32(12)  # [0, 2^20)
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**20 - 1, nb, what=f"nb={nb}",
           use_bucket_oracle=nb >= 4096)


def test_min_equals_max_and_narrow_ranges(rs, oracle):
    keys = np.full(100_000, 77, np.uint32)
    _check(rs, oracle, keys, synth.index_values(keys.size), 77, 77, 0, what="min==max")
    keys = synth.uniform_below(200_000, 3, 5, 52) + np.uint32(10)
    _check(rs, oracle, keys, synth.index_values(keys.size), 10, 12, 0, what="range 3")
    _check(rs, oracle, keys, synth.index_values(keys.size), 0, 2**32 - 1, 7, what="range 3 nb 7",
           use_bucket_oracle=False)


def test_skewed_keys_take_the_overflow_path(rs, oracle):
    """Gaussian keys under the full declared range [0, 2^32): most keys fall in
    a few buckets, which are sorted by the radix of their key range."""
    n = 2_000_000
    keys = synth.gaussian_u32(n, seed=9)
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**32 - 1, n // 16, what="gaussian", use_bucket_oracle=False)
    few = np.array([5, 2**31, 2**32 - 1], np.uint32)[synth.uniform_below(n, 3, 9, 53)]
    _check(rs, oracle, few, synth.index_values(n), 0, 2**32 - 1, 0, what="three values", use_bucket_oracle=False)


@pytest.mark.parametrize("key_bits", [40, 64])
def test_u64(rs, oracle, key_bits):
    n = 300_001
    keys = synth.keys_u64(n, key_bits, seed=key_bits)
    vals = synth.index_values(n)
    _check(rs, oracle, keys, vals, 0, 2**key_bits - 1, 0, what=f"u64 {key_bits}", use_bucket_oracle=False)
    _check(rs, oracle, keys, vals, None, None, 0, what=f"u64 {key_bits} computed", use_bucket_oracle=False)
    small = synth.keys_u64(50_000, key_bits, seed=1)
    _check(rs, oracle, small, synth.index_values(small.size), 0, 2**key_bits - 1, 0, what="u64 vs bucket oracle")


@pytest.mark.parametrize("key_bits", [40, 50])
def test_u64_equal_keys_within_buckets(rs, oracle, key_bits):
    """64-bit keys drawn from n/2.5 distinct values, so buckets of ~16 keys
    hold equal keys: the rank sort of every bucket must keep them in input
    order (their values show it).  40- and 50-bit keys make runs of buckets
    narrow enough for the rank sort's one-comparison form (key bits + 12 of
    position within 64)."""
    n = 300_000
    distinct = synth.keys_u64(120_000, key_bits, seed=key_bits + 7)
    keys = distinct[synth.uniform_below(n, distinct.size, key_bits, 54)]
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**key_bits - 1, 0, what=f"u64 dup {key_bits}",
           use_bucket_oracle=False)
    small = keys[:60_000].copy()
    _check(rs, oracle, small, synth.index_values(small.size), 0, 2**key_bits - 1, 0,
           what=f"u64 dup {key_bits} vs bucket oracle")


def test_in_place(rs, oracle):
    n = 250_000
    keys = synth.u32(n, 54, 0)
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**32 - 1, 0, in_place=True, what="in place",
           use_bucket_oracle=False)


def test_key_outside_declared_range_is_reported(rs):
    import torch

    keys = synth.u32(10_000, 55, 0) >> np.uint32(16)
    keys[5] = 70_000
    kd = to_dev(keys)
    out = torch.empty_like(kd)
    ws = rs.workspace(rs.rs_workspace_bytes(1, 4, 0, keys.size, 0, 0, 0))
    assert rs.bs_sort_u32(kd, out, None, None, keys.size, 0, 65_535, 0, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE


@pytest.mark.slow
@pytest.mark.parametrize("dist", [0, 1, 2, 3, 4, 5, 6])
def test_full_size_100m(rs, oracle, dist):
    """100M u32 keys of every benchmark distribution (uniform, small range,
    large range, sorted, reverse, nearly sorted, Gaussian) with their declared
    bounds and n/16 buckets, checked in full against the oracle radix sort."""
    import torch

    n = 100_000_000
    keys = synth.keys_u32(n, dist, seed=0)
    lo, hi = synth.DECLARED_BOUNDS[dist]
    gk, _ = _bucket(rs, keys, None, lo, hi, 0)
    torch.cuda.empty_cache()
    assert_same(gk, oracle.radix_sort(keys), f"100M {synth.DISTS[dist]}")


def _edge_keys(lo, hi, nb, count, seed, dtype):
    """Keys uniform in [lo, hi] plus the keys next to bucket boundaries: the
    first key of bucket b is lo + ceil(b * R / nb), R = hi - lo + 1."""
    R = hi - lo + 1
    if R <= 2**32:
        body = [lo + int(x) for x in synth.uniform_below(count, R, seed, 70)] if R < 2**32 else \
            [lo + int(x) for x in synth.u32(count, seed, 70)]
    else:
        body = [lo + (int(x) % R) for x in synth.u64(count, seed, 70)]
    edges = []
    for b in [0, 1, 2, nb // 3, nb // 2, nb - 2, nb - 1] + [int(x) for x in synth.uniform_below(64, nb, seed, 71)]:
        if 0 <= b < nb:
            first = lo + -(-b * R // nb)
            edges += [first - 1, first, first + 1]
    edges = [e for e in edges if lo <= e <= hi] + [lo, hi]
    return np.array(body + edges, dtype=dtype)


@pytest.mark.parametrize("kb,lo,hi,nb", [
    (4, 0, 2**32 - 1, 6_250_000), (4, 0, 2**31 - 1, 62_500), (4, 10, 12, 7), (4, 5, 5, 1),
    (4, 0, 2**20 - 1, 300_000), (4, 1000, 10**9, 3), (4, 123, 2**32 - 1, 2**20 + 7), (4, 0, 999, 1000),
    (8, 0, 2**64 - 1, 12_345), (8, 0, 2**40 - 1, 1 << 22), (8, 7, 2**63, 2**20), (8, 2**63, 2**63 + 5, 9)])
def test_bucket_counts_are_exact(rs, oracle, kb, lo, hi, nb):
    """b(k) = floor((k - min) * nb / (max - min + 1)) on the GPU, checked
    bucket by bucket against the oracle's counts, with keys on both sides of
    bucket boundaries."""
    import torch

    dt = np.uint32 if kb == 4 else np.uint64
    keys = _edge_keys(lo, hi, nb, 200_000, 17 + nb % 89, dt)
    kd = to_dev(keys)
    counts = torch.empty(nb, dtype=torch.int32, device="cuda")
    ws = rs.workspace(4096)
    fn = rs.bs_bucket_counts_u32 if kb == 4 else rs.bs_bucket_counts_u64
    assert fn(kd, keys.size, lo, hi, nb, counts, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 0
    got = from_dev(counts, np.uint32).astype(np.uint64)
    assert_same(got, oracle.bucket_counts(keys, lo, hi, nb), f"counts kb={kb} [{lo},{hi}] nb={nb}")


def test_bucket_counts_report_keys_outside_the_range(rs):
    import torch

    keys = np.array([5, 6, 7, 100, 8], np.uint32)
    counts = torch.empty(4, dtype=torch.int32, device="cuda")
    ws = rs.workspace(4096)
    assert rs.bs_bucket_counts_u32(to_dev(keys), 5, 5, 8, 4, counts, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE
    assert from_dev(counts, np.uint32).tolist() == [1, 1, 1, 1]


@pytest.mark.parametrize("n,nb", [(1000, 0), (4000, 200), (100_000, 1), (100_000, 2), (3000, 1)])
def test_u64_full_range_small_bucket_counts(rs, oracle, n, nb):
    """64-bit keys over the whole range [0, 2^64 - 1] with few buckets: a
    group of buckets (or one bucket) then covers all 2^64 key values, a
    width that only fits 64 bits as width - 1."""
    keys = synth.keys_u64(n, 64, seed=n + nb)
    keys[:2] = [0, 2**64 - 1]
    _check(rs, oracle, keys, synth.index_values(n), 0, 2**64 - 1, nb, what=f"u64 full n={n} nb={nb}",
           use_bucket_oracle=False)


@pytest.mark.parametrize("nb,lo,hi", [(125_000, 0, 2**32 - 1), ((1 << 22) + 12_345, 0, 2**32 - 1),
                                      (300_007, 17, 3_000_000_017)])
def test_bucket_ids_at_partition_boundaries(rs, oracle, nb, lo, hi):
    """Keys at the first key of buckets whose id is a multiple of a partition
    level's 2^shift (and the key just below): there the cheap bucket-id
    estimate and the exact id can differ in the partition digit, and the
    remainder test must run.  Level shifts as the sort plans them (8-bit
    digits from the top of the bucket id)."""
    R = hi - lo + 1
    bbits = (nb - 1).bit_length()
    d1 = min(8, bbits)
    s1 = bbits - d1
    s2 = s1 - min(8, s1)
    bs = sorted(set(range(0, nb, 1 << s1)) | set(range(0, nb, 1 << s2)))
    first = np.array([lo + (b * R + nb - 1) // nb for b in bs], dtype=np.uint64)
    edge = np.concatenate([first, first[first > lo] - np.uint64(1)]).astype(np.uint32)
    rest = (synth.u64(400_000, 610, 0) % np.uint64(R) + np.uint64(lo)).astype(np.uint32)
    keys = np.concatenate([edge, rest])
    keys = keys[synth.u64(keys.size, 611, 0).argsort(kind="stable")]  # mixed order
    _check(rs, oracle, keys, synth.index_values(keys.size), lo, hi, nb, what=f"boundaries nb={nb}")
