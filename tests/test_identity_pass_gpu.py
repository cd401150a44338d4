"""GPU parity of passes whose keys all carry one digit.  Such a pass keeps the
input order (the counting sort places the keys of one digit in input order),
and the scatter kernel then copies its input instead of ranking it.  These
cases put identity passes first, last, in the middle and everywhere, for
plain and typed keys, with and without values, in place and not, and
compare with the oracle bit for bit."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu

N = 300_001  # well above one block's shared-memory sort, with a ragged last tile


def _radix(rs, oracle, keys, vals=None, key_bits=0, in_place=False, what=""):
    import torch

    kbits = key_bits or 8 * keys.dtype.itemsize
    k = to_dev(keys)
    v = to_dev(vals) if vals is not None else None
    if in_place:
        out, outv = rs.sort(k, v, key_bits, out=k, out_values=v)
    else:
        out, outv = rs.sort(k, v, key_bits)
    torch.cuda.synchronize()
    if vals is None:
        assert_same(from_dev(out, keys.dtype), oracle.radix_sort(keys, None, kbits), what)
    else:
        wk, wv = oracle.radix_sort(keys, vals, kbits)
        assert_same(from_dev(out, keys.dtype), wk, what + " keys")
        assert_same(from_dev(outv, np.uint32), wv, what + " values")


@pytest.mark.parametrize("with_values", [False, True])
@pytest.mark.parametrize("in_place", [False, True])
def test_u32_identity_passes(rs, oracle, with_values, in_place):
    vals = synth.index_values(N) if with_values else None
    u = synth.u32(N, 601, 0)
    # passes 1..3 identity (keys < 256), then pass 0 identity (low byte fixed),
    # then the two middle passes identity, then every pass (one key repeated)
    cases = {
        "keys below 256": u & np.uint32(0xFF),
        "constant low byte": (u & np.uint32(0xFFFFFF00)) | np.uint32(0x5A),
        "constant middle bytes": (u & np.uint32(0xFF0000FF)) | np.uint32(0x00ABCD00),
        "one repeated key": np.full(N, 0xDEADBEEF, np.uint32),
    }
    for what, keys in cases.items():
        _radix(rs, oracle, keys, vals, 0, in_place, what)


def test_u32_identity_passes_with_trimmed_key_bits(rs, oracle):
    keys = synth.u32(N, 602, 0) & np.uint32(0x000F00FF)  # 24 bits: pass 1 identity, 3 passes
    _radix(rs, oracle, keys, None, 24, what="24-bit keys, middle pass identity")
    _radix(rs, oracle, keys, synth.index_values(N), 24, in_place=True, what="24-bit keys in place")


@pytest.mark.parametrize("with_values", [False, True])
def test_u64_identity_passes(rs, oracle, with_values):
    vals = synth.index_values(N) if with_values else None
    keys = synth.keys_u64(N, 32, seed=603)  # the upper four passes are identities
    _radix(rs, oracle, keys, vals, 64, what="u64 keys below 2^32")
    keys = synth.keys_u64(N, 64, seed=604) & np.uint64(0xFFFF00000000FFFF)
    _radix(rs, oracle, keys, vals, 64, in_place=True, what="u64 keys with zero middle bytes")


@pytest.mark.parametrize("dt,desc", [(np.int32, False), (np.int32, True), (np.float32, False),
                                     (np.float64, True)])
def test_typed_identity_passes(rs, oracle, dt, desc):
    """Small non-negative integers (as int or float): the ordered images share
    their high bytes, and small integers as floats have zero low mantissa
    bytes, so the first and the last pass (which carry the typed-key mapping)
    are identities."""
    import torch

    ints = (synth.u32(N, 605, 0) % np.uint32(1000)).astype(np.int64)
    x = ints.astype(dt)
    ut = {4: np.uint32, 8: np.uint64}[x.dtype.itemsize]
    kind = 2 if np.issubdtype(dt, np.floating) else 1
    vals = synth.index_values(N)
    signed = {4: np.int32, 8: np.int64}[x.dtype.itemsize]
    kd = torch.from_numpy(np.ascontiguousarray(x).view(signed)).cuda()
    vd = to_dev(vals)
    ok, ov = rs.sort_typed(kd, vd, kind=kind, descending=desc)
    torch.cuda.synchronize()
    wk, wv = oracle.sort_typed(x, vals, kind, desc)
    assert_same(ok.cpu().numpy().view(ut), wk.view(ut), f"{dt.__name__} desc={desc} keys")
    assert_same(ov.cpu().numpy().view(np.uint32), wv, f"{dt.__name__} desc={desc} values")


def test_bucket_identity_level_pass(rs, oracle):
    """Keys in [0, 1000) under declared bounds [0, 2^32 - 1]: every key falls
    in the first level-1 digit of the bucket id, so that pass is an identity."""
    import torch

    keys = synth.keys_u32(N, 1, seed=606)
    vals = synth.index_values(N)
    nb = N // 16
    kd, vd = to_dev(keys), to_dev(vals)
    ok, ov = rs.bucket_sort(kd, vd, min_key=0, max_key=2**32 - 1, num_buckets=nb)
    torch.cuda.synchronize()
    wk, wv = oracle.bucket_sort(keys, vals, 0, 2**32 - 1, nb)
    assert_same(from_dev(ok, np.uint32), wk, "bucket keys")
    assert_same(from_dev(ov, np.uint32), wv, "bucket values")


def test_counting_pass_on_a_constant_digit(rs, oracle):
    """The counting-sort building block on a digit every key shares returns
    its input unchanged."""
    import torch

    keys = (synth.u32(N, 607, 0) & np.uint32(0xFFFF00FF)) | np.uint32(0x3C00)
    vals = synth.index_values(N)
    ok, ov = rs.counting_pass(to_dev(keys), to_dev(vals), shift=8, digit_bits=8)
    torch.cuda.synchronize()
    wk, wv = oracle.counting_pass(keys, vals, 8, 8)
    assert_same(wk, keys, "oracle: identity")
    assert_same(from_dev(ok, np.uint32), wk, "identity counting pass keys")
    assert_same(from_dev(ov, np.uint32), wv, "identity counting pass values")


# Warps whose keys all carry one digit (runs of sorted keys) skip the ranking:
# each key's rank is its position in the warp.  The cases below make such
# warps in some passes but not others, with values so that order shows.

def _runs_of_top_digit(n, seed, width=32):
    """Keys grouped by their top byte in runs of about 600, random below it."""
    top = (np.arange(n, dtype=np.uint64) // np.uint64(600)) % np.uint64(256)
    if width == 32:
        low = synth.u32(n, seed, 0) & np.uint32(0x00FFFFFF)
        return ((top.astype(np.uint32) << np.uint32(24)) | low).astype(np.uint32)
    low = synth.keys_u64(n, 56, seed=seed)
    return (top << np.uint64(56)) | low


@pytest.mark.parametrize("with_values", [False, True])
def test_warp_uniform_digits_u32(rs, oracle, with_values):
    n = 1_000_003
    vals = synth.index_values(n) if with_values else None
    _radix(rs, oracle, _runs_of_top_digit(n, 620), vals, what="runs of one top digit")
    s = np.sort(synth.u32(n, 621, 0))
    _radix(rs, oracle, s, vals, what="sorted keys")
    dup = np.repeat(synth.u32(n // 700 + 1, 622, 0), 700)[:n]  # long runs of one key
    _radix(rs, oracle, dup, vals, in_place=True, what="runs of one key, in place")
    _radix(rs, oracle, s[::-1].copy(), vals, key_bits=32, what="reverse sorted keys")


def test_warp_uniform_digits_u64_and_typed(rs, oracle):
    import torch

    n = 700_001
    vals = synth.index_values(n)
    _radix(rs, oracle, _runs_of_top_digit(n, 623, 64), vals, what="u64 runs of one top digit")
    x = np.sort(synth.u32(n, 624, 0).view(np.int32))
    kd = torch.from_numpy(x.copy()).cuda()
    ok, ov = rs.sort_typed(kd, to_dev(vals), kind=1)
    torch.cuda.synchronize()
    wk, wv = oracle.sort_typed(x, vals, 1, False)
    assert_same(ok.cpu().numpy().view(np.uint32), wk.view(np.uint32), "typed sorted int32 keys")
    assert_same(ov.cpu().numpy().view(np.uint32), wv, "typed sorted int32 values")


def test_warp_uniform_digits_segmented_and_bucket(rs, oracle):
    import torch

    sizes = synth.log_uniform_sizes(60, 5000, 300_000, seed=625)
    n = int(sizes.sum())
    keys = _runs_of_top_digit(n, 626)
    vals = synth.index_values(n)
    off = synth.segment_offsets(sizes)
    kd, vd, od = to_dev(keys), to_dev(vals), to_dev(off.astype(np.uint64))
    ok, ov = rs.segmented_sort(kd, od, vd)
    torch.cuda.synchronize()
    wk, wv = oracle.segmented_radix_sort(keys, off, vals, 32)
    assert_same(from_dev(ok, np.uint32), wk, "segmented keys")
    assert_same(from_dev(ov, np.uint32), wv, "segmented values")
    s = np.sort(synth.u32(n, 627, 0))
    ok, ov = rs.bucket_sort(to_dev(s), vd)
    torch.cuda.synchronize()
    wk, wv = oracle.bucket_sort(s, vals, int(s.min()), int(s.max()), max(1, n // 16))
    assert_same(from_dev(ok, np.uint32), wk, "bucket sorted keys")
    assert_same(from_dev(ov, np.uint32), wv, "bucket sorted values")


# Segments sorted in shared memory (up to 4096 keys) whose keys are already in
# nondecreasing order are written back as loaded.  The cases mix such segments
# with near misses (one pair out of order at either end).

@pytest.mark.parametrize("kb", [4, 8])
def test_already_sorted_small_segments(rs, oracle, kb):
    import torch

    sizes = synth.log_uniform_sizes(400, 2, 4096, seed=631)
    n = int(sizes.sum())
    off = synth.segment_offsets(sizes)
    keys = synth.u32(n, 630, 0) if kb == 4 else synth.keys_u64(n, 64, seed=630)
    for s_ in range(len(sizes)):
        a, b = int(off[s_]), int(off[s_ + 1])
        seg = np.sort(keys[a:b])
        mode = s_ % 5
        if mode == 1 and b - a >= 2:
            seg[-2], seg[-1] = seg[-1], seg[-2]   # one inversion at the end
        elif mode == 2 and b - a >= 2:
            seg[0], seg[1] = seg[1], seg[0]       # one inversion at the start
        elif mode == 3:
            seg[:] = seg[0]                       # all equal
        elif mode == 4:
            seg = seg[::-1].copy()                # descending
        keys[a:b] = seg
    vals = synth.index_values(n)
    kd, vd, od = to_dev(keys), to_dev(vals), to_dev(off.astype(np.uint64))
    ok, ov = rs.segmented_sort(kd, od, vd)
    torch.cuda.synchronize()
    wk, wv = oracle.segmented_radix_sort(keys, off, vals, 8 * kb)
    assert_same(from_dev(ok, keys.dtype), wk, "sorted-run segments keys")
    assert_same(from_dev(ov, np.uint32), wv, "sorted-run segments values")


def test_already_sorted_single_block_sorts(rs, oracle):
    import torch

    for n, kind in ((4096, "sorted"), (4000, "equal"), (3000, "last pair swapped"), (1, "one key")):
        keys = np.sort(synth.u32(n, 632, 0))
        if kind == "equal":
            keys[:] = 7
        elif kind == "last pair swapped" and n >= 2:
            keys[-2], keys[-1] = keys[-1], keys[-2]
        _radix(rs, oracle, keys, synth.index_values(n), what=f"one block, {kind}")
    # typed keys in order: floats with negatives, sorted by value
    x = np.sort((synth.unit_doubles(3000, 633, 0) * 2 - 1).astype(np.float32))
    vals = synth.index_values(3000)
    kd = torch.from_numpy(x.view(np.int32).copy()).cuda()
    ok, ov = rs.sort_typed(kd, to_dev(vals), kind=2)
    torch.cuda.synchronize()
    wk, wv = oracle.sort_typed(x, vals, 2, False)
    assert_same(ok.cpu().numpy().view(np.uint32), wk.view(np.uint32), "typed floats in order")
    assert_same(ov.cpu().numpy().view(np.uint32), wv, "typed floats in order, values")


# A radix sort whose input is already in order (the count kernel checks every
# key against its successor) returns the input: the passes return at once and
# the last copies the input to the output.

@pytest.mark.parametrize("with_values", [False, True])
def test_radix_of_input_already_in_order(rs, oracle, with_values):
    n = 1_000_003
    vals = synth.index_values(n) if with_values else None
    keys = np.sort(synth.u32(n, 640, 0) >> np.uint32(8))  # repeated keys, so order of equals shows
    _radix(rs, oracle, keys, vals, what="in order")
    _radix(rs, oracle, keys, vals, in_place=True, what="in order, in place (4 passes)")
    _radix(rs, oracle, keys >> np.uint32(8), vals, key_bits=24, in_place=True, what="in order, in place (3 passes)")
    miss = keys.copy()
    miss[-1] = miss[-2] - np.uint32(1)                        # one pair out of order at the end
    _radix(rs, oracle, miss, vals, what="out of order at the end")
    miss = keys.copy()
    miss[0] = miss[1] + np.uint32(1)                          # and at the start
    _radix(rs, oracle, miss, vals, what="out of order at the start")
    _radix(rs, oracle, np.sort(synth.keys_u64(n, 64, seed=641)), synth.index_values(n), what="u64 in order")


def test_typed_input_already_in_order(rs, oracle):
    import torch

    n = 500_001
    vals = synth.index_values(n)
    x = np.sort((synth.unit_doubles(n, 642, 0) * 2e6 - 1e6).astype(np.float32))
    for desc, arr in ((False, x), (True, x[::-1].copy())):   # in order for the requested direction
        kd = torch.from_numpy(arr.view(np.int32).copy()).cuda()
        ok, ov = rs.sort_typed(kd, to_dev(vals), kind=2, descending=desc)
        torch.cuda.synchronize()
        wk, wv = oracle.sort_typed(arr, vals, 2, desc)
        assert_same(ok.cpu().numpy().view(np.uint32), wk.view(np.uint32), f"typed in order desc={desc}")
        assert_same(ov.cpu().numpy().view(np.uint32), wv, f"typed in order desc={desc} values")


def test_plan_replay_alternating_in_order_and_not(rs, oracle):
    """The verdict is taken afresh on every call: a plan replayed on ordered
    and then on unordered keys in the same buffer sorts both."""
    import torch

    n = 2_000_000
    kd = to_dev(synth.u32(n, 643, 0))
    ok = torch.empty_like(kd)
    plan = rs.Plan(rs.RS_PLAN_RADIX, kd, ok)
    for rep in range(2):
        for keys in (np.sort(synth.u32(n, 644 + rep, 0)), synth.u32(n, 646 + rep, 0)):
            kd.copy_(to_dev(keys))
            plan.launch()
            torch.cuda.synchronize()
            assert_same(from_dev(ok, np.uint32), np.sort(keys), f"replay {rep}")
    plan.close()
