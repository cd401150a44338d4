"""GPU parity of the segmented sort: every segment must equal the oracle's
sort of that segment alone (keys and values, zero tolerance)."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _run(rs, keys, sizes, vals=None, key_bits=0, in_place=False):
    import torch

    off = synth.segment_offsets(sizes)
    kd = to_dev(keys)
    vd = to_dev(vals) if vals is not None else None
    od = to_dev(off.astype(np.uint64))
    if in_place:
        ok, ov = rs.segmented_sort(kd, od, vd, key_bits, out=kd, out_values=vd)
    else:
        ok, ov = rs.segmented_sort(kd, od, vd, key_bits)
    torch.cuda.synchronize()
    return off, from_dev(ok, keys.dtype), (from_dev(ov, np.uint32) if vals is not None else None)


def _check(rs, oracle, keys, sizes, vals=None, key_bits=0, in_place=False, what=""):
    kbits = key_bits or 8 * keys.dtype.itemsize
    off, gk, gv = _run(rs, keys, sizes, vals, key_bits, in_place)
    if vals is None:
        want = oracle.segmented_radix_sort(keys, off, None, kbits)
        assert_same(gk, want, what)
    else:
        wk, wv = oracle.segmented_radix_sort(keys, off, vals, kbits)
        assert_same(gk, wk, what + " keys")
        assert_same(gv, wv, what + " values")


# tiny-sort and shared-memory-sort limits (256, 4096), the shared-memory
# sort's switch between 4 and 16 keys per lane (1024), its whole-warp runs
# (multiples of 128 and 512 keys), tile edges of the scatter passes
EDGE_SIZES = [0, 1, 2, 3, 0, 255, 256, 4095, 4096, 4097, 4608, 4609, 6143, 6144, 6145, 9217, 12289, 70_001, 0, 1,
              3072, 3073, 200_000, 257, 383, 384, 385, 511, 512, 513, 1023, 1024, 1025, 1535, 1536, 1537, 2047,
              2048, 2049, 3583, 3584, 3585]


@pytest.mark.parametrize("kb,with_values", [(4, False), (4, True), (8, False), (8, True)])
def test_segment_size_edges(rs, oracle, kb, with_values):
    n = sum(EDGE_SIZES)
    keys = synth.u32(n, 40, 0) if kb == 4 else synth.keys_u64(n, 64, seed=41)
    vals = synth.index_values(n) if with_values else None
    _check(rs, oracle, keys, EDGE_SIZES, vals, what=f"edges kb={kb} v={with_values}")


def test_log_uniform_batch_like_the_batched_workload(rs, oracle):
    """300 arrays with sizes log-uniform in [256, 200000] (the batched
    workload's size law, scaled down), uniform u32 keys."""
    sizes = synth.log_uniform_sizes(300, 256, 200_000, seed=0)
    n = int(sizes.sum())
    keys = synth.u32(n, 42, 0)
    _check(rs, oracle, keys, sizes, None, what="log-uniform")
    _check(rs, oracle, keys, sizes, synth.index_values(n), what="log-uniform kv")


@pytest.mark.parametrize("dist", [1, 3, 4, 6, 8])
def test_distributions(rs, oracle, dist):
    sizes = [5000, 300, 100_000, 4096, 17]
    n = sum(sizes)
    keys = synth.keys_u32(n, dist, seed=dist)
    _check(rs, oracle, keys, sizes, synth.index_values(n), what=synth.DISTS[dist])


@pytest.mark.parametrize("key_bits", [1, 12, 24, 31])
def test_key_bits(rs, oracle, key_bits):
    sizes = [10_000, 3000, 50_000]
    n = sum(sizes)
    keys = synth.u32(n, 43 + key_bits, 0) >> np.uint32(32 - key_bits)
    _check(rs, oracle, keys, sizes, synth.index_values(n), key_bits, what=f"key_bits {key_bits}")


@pytest.mark.parametrize("key_bits", [32, 24])
def test_in_place(rs, oracle, key_bits):
    sizes = [7000, 100, 60_000, 0, 4096]
    n = sum(sizes)
    keys = synth.u32(n, 44, 0) >> np.uint32(32 - key_bits)
    _check(rs, oracle, keys, sizes, synth.index_values(n), key_bits, in_place=True, what=f"in place {key_bits}")


def test_single_segment_equals_plain_sort(rs, oracle):
    n = 1_000_003
    keys = synth.u32(n, 45, 0)
    _check(rs, oracle, keys, [n], None, what="one segment")


def test_bad_offsets_are_reported(rs):
    import torch

    keys = to_dev(synth.u32(100, 46, 0))
    off = to_dev(np.array([0, 50, 40, 100], np.uint64))  # decreasing
    ws = rs.workspace(rs.rs_segmented_workspace_bytes(4, 0, 100, 3, 32))
    out = torch.empty_like(keys)
    assert rs.rs_sort_segmented_u32(keys, out, None, None, off, 3, 100, 32, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 1  # RS_ERR_INVALID_ARG recorded on the device


@pytest.mark.parametrize("past", [1, 5000])
def test_offsets_past_n_total_are_reported_and_nothing_is_written_outside(rs, oracle, past):
    """An offsets table that ends past n_total: the segment that runs past it
    is dropped and reported as RS_ERR_INVALID_ARG, the segments inside are
    still sorted, and guard words around the output and after the workspace
    are unchanged (no write outside the arrays)."""
    import torch

    sizes = [3000, 70_000, 100]
    n = sum(sizes)
    keys = synth.u32(n, 48, 0)
    off = synth.segment_offsets(sizes).astype(np.uint64)
    off[-1] = n + past  # the last segment ends past n_total
    G = 1 << 16
    guard = -0x21524111  # 0xdeadbeef as int32
    kd = to_dev(keys)
    out = torch.full((n + 2 * G,), guard, dtype=torch.int32, device="cuda")
    wsb = rs.rs_segmented_workspace_bytes(4, 0, n, 3, 32)
    wsbuf = torch.full((wsb + G,), 0x5A, dtype=torch.uint8, device="cuda")
    ws = wsbuf[:wsb]
    assert rs.rs_sort_segmented_u32(kd, out[G:G + n], None, None, to_dev(off), 3, n, 32, ws, wsb) == 0
    assert rs.get_status(ws) == 1  # RS_ERR_INVALID_ARG
    o = out.cpu().numpy()
    assert np.all(o[:G] == guard) and np.all(o[G + n:] == guard)
    assert np.all(wsbuf[wsb:].cpu().numpy() == 0x5A)
    got = o[G:G + n].view(np.uint32)
    for a, b in [(0, 3000), (3000, 73_000)]:  # the segments inside n_total are sorted
        assert_same(got[a:b], oracle.radix_sort(keys[a:b]), f"segment [{a},{b})")


def test_key_above_key_bits_in_a_large_segment_is_reported(rs):
    import torch

    sizes = [100, 20_000, 300]
    n = sum(sizes)
    keys = synth.u32(n, 49, 0) >> np.uint32(20)  # 12-bit keys
    keys[5_000] = 1 << 12  # inside the scatter-pass segment
    kd = to_dev(keys)
    off = to_dev(synth.segment_offsets(sizes))
    ws = rs.workspace(rs.rs_segmented_workspace_bytes(4, 0, n, 3, 12))
    out = torch.empty_like(kd)
    assert rs.rs_sort_segmented_u32(kd, out, None, None, off, 3, n, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE


def test_key_above_key_bits_in_a_small_segment_is_reported(rs):
    import torch

    sizes = [100, 20_000, 300]
    n = sum(sizes)
    keys = synth.u32(n, 47, 0) >> np.uint32(20)  # 12-bit keys
    keys[20_150] = 1 << 12  # inside the last (shared-memory) segment
    kd = to_dev(keys)
    off = to_dev(synth.segment_offsets(sizes))
    ws = rs.workspace(rs.rs_segmented_workspace_bytes(4, 0, n, 3, 12))
    out = torch.empty_like(kd)
    assert rs.rs_sort_segmented_u32(kd, out, None, None, off, 3, n, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE


def _u32_as_i64(t):
    return t.to(__import__("torch").int64) & 0xFFFFFFFF


@pytest.mark.slow
def test_full_batched_workload_sampled_against_oracle(rs, oracle):
    """The batched workload at full size, in the launch configuration the
    benchmark times (a segmented-sort plan replayed from a CUDA graph):
    20,000 uint32 arrays with sizes log-uniform in [256, 2,000,000], about
    4.5e9 keys, so offsets pass 2^32.  Every 100th array, every array above
    1M keys (about 1,500 of them, half the keys) and the edge arrays
    (including the last, past 2^32) are compared element by element with the
    oracle; every array is also checked on the device to be nondecreasing
    with its key sum and sum of squares (mod 2^64) unchanged."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    import torch

    sizes = synth.log_uniform_sizes(20_000, 256, 2_000_000, seed=0)
    off = synth.segment_offsets(sizes)
    n = int(off[-1])
    assert n > 2**32
    kd = synth.u32_torch(n, seed=0, dist_id=0, device="cuda")
    od = torch.from_numpy(off.view(np.int64)).cuda()
    out = torch.empty_like(kd)
    plan = rs.Plan(rs.RS_PLAN_SEGMENTED, kd, out, seg_offsets=od)
    out.zero_()
    plan.launch()
    torch.cuda.synchronize()
    assert rs.get_status(plan.ws) == 0
    sample = set(range(0, sizes.size, 100)) | set(np.flatnonzero(sizes > 1_000_000).tolist())
    sample |= {1, 777, 19_998, 19_999, int(np.argmax(sizes)), int(np.argmin(sizes))}
    sample = sorted(sample)
    assert len(sample) > 1000

    def compare(i):
        # the oracle's C routine runs without the GIL, so arrays are checked
        # on several host threads at once
        a, b = int(off[i]), int(off[i + 1])
        keys = kd[a:b].cpu().numpy().view(np.uint32)
        got = out[a:b].cpu().numpy().view(np.uint32)
        assert_same(got, oracle.radix_sort(keys, None, 32), f"array {i}")
        return b - a

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        checked = sum(ex.map(compare, sample))
    assert checked > n // 3
    # properties of every array, in chunks of whole arrays
    starts = torch.from_numpy(off[:-1].view(np.int64)).cuda()
    i0 = 0
    while i0 < sizes.size:
        i1 = int(np.searchsorted(off, off[i0] + (1 << 28), side="right")) - 1
        i1 = max(i1, i0 + 1)
        a, b = int(off[i0]), int(off[i1])
        x, y = _u32_as_i64(kd[a:b]), _u32_as_i64(out[a:b])
        step_ok = y[1:] >= y[:-1]
        step_ok[(starts[i0 + 1:i1] - a - 1)] = True  # array boundaries
        assert bool(step_ok.all()), f"arrays {i0}..{i1} not sorted"
        seg = torch.repeat_interleave(torch.arange(i1 - i0, device="cuda"),
                                      torch.from_numpy(sizes[i0:i1]).cuda())
        for f in (lambda v: v, lambda v: v * v):
            sx = torch.zeros(i1 - i0, dtype=torch.int64, device="cuda").index_add_(0, seg, f(x))
            sy = torch.zeros(i1 - i0, dtype=torch.int64, device="cuda").index_add_(0, seg, f(y))
            assert torch.equal(sx, sy), f"arrays {i0}..{i1}: multiset changed"
        i0 = i1
    plan.close()


@pytest.mark.parametrize("kb,with_values", [(4, False), (4, True), (8, False), (8, True)])
def test_every_compiled_shape_gives_identical_bits(rs, oracle, kb, with_values):
    """rs_sort_segmented_*_ex with each kernel shape compiled for segmented
    passes (every radix shape at 8-bit digits): the same bits as the oracle;
    another digit width is refused."""
    import torch

    sizes = [70_001, 5000, 4097, 300, 12_289, 0, 40_000]
    n = sum(sizes)
    keys = synth.u32(n, 48, 0) if kb == 4 else synth.keys_u64(n, 64, seed=48)
    vals = synth.index_values(n) if with_values else None
    off = synth.segment_offsets(sizes)
    kd, od = to_dev(keys), to_dev(off.astype(np.uint64))
    vd = to_dev(vals) if with_values else None
    ws = rs.workspace(rs.rs_segmented_workspace_bytes(kb, with_values, n, len(sizes), 0))
    fn = rs.rs_sort_segmented_u32_ex if kb == 4 else rs.rs_sort_segmented_u64_ex
    want = oracle.segmented_radix_sort(keys, off, vals, 8 * kb)
    shapes = sorted({rs.rs_config_get(kb, with_values, i).as_tuple()[1:]
                     for i in range(rs.rs_config_count(kb, with_values))})
    assert len(shapes) >= 2
    for block, items in shapes:
        ok = torch.empty_like(kd)
        ov = torch.empty_like(vd) if with_values else None
        assert fn(kd, ok, vd, ov, od, len(sizes), n, 0, ws, ws.numel(), None, (8, block, items)) == 0
        torch.cuda.synchronize()
        assert rs.get_status(ws) == 0
        if with_values:
            assert_same(from_dev(ok, keys.dtype), want[0], f"{block}x{items} keys")
            assert_same(from_dev(ov, np.uint32), want[1], f"{block}x{items} values")
        else:
            assert_same(from_dev(ok, keys.dtype), want, f"{block}x{items}")
    ok = torch.empty_like(kd)
    ov = torch.empty_like(vd) if with_values else None
    assert fn(kd, ok, vd, ov, od, len(sizes), n, 0, ws, ws.numel(), None, (7,) + shapes[0]) == 9  # UNSUPPORTED


@pytest.mark.parametrize("kb,with_values,in_place", [(4, False, False), (4, True, True), (8, False, True),
                                                     (8, True, False)])
def test_many_tiny_segments(rs, oracle, kb, with_values, in_place):
    """Thousands of segments of 0..256 keys (sorted one warp each) mixed with
    a few larger ones, with repeated keys so that stability shows."""
    sizes = synth.uniform_below(6000, 257, 90 + kb, 91).astype(np.int64)
    sizes[::500] = 5000  # a few shared-memory segments
    sizes[7] = 20_000    # and a scatter-pass one
    n = int(sizes.sum())
    keys = (synth.u32(n, 92, 0) >> np.uint32(26)) if kb == 4 else (synth.keys_u64(n, 64, seed=92) >> np.uint64(58))
    vals = synth.index_values(n) if with_values else None
    _check(rs, oracle, keys, sizes, vals, in_place=in_place, what=f"tiny kb={kb} v={with_values} ip={in_place}")


@pytest.mark.parametrize("kb", [4, 8])
def test_tiny_segments_holding_the_largest_key(rs, oracle, kb):
    """Warp-sorted segments whose keys are the largest value of the key type
    (which also pads the sorting network past the segment's end) or one below
    it: the largest keys stay in the segment, in input order."""
    sizes = np.array([33, 64, 65, 100, 128, 129, 200, 256, 255, 31, 1, 0, 77] * 40, dtype=np.int64)
    n = int(sizes.sum())
    top = np.uint32(0xFFFFFFFF) if kb == 4 else np.uint64(0xFFFFFFFFFFFFFFFF)
    bit = synth.u32(n, 94, 0) & np.uint32(1)
    keys = (top - bit.astype(top.dtype)).astype(top.dtype)
    for with_values in (False, True):
        vals = synth.index_values(n) if with_values else None
        _check(rs, oracle, keys, sizes, vals, what=f"largest keys kb={kb} v={with_values}")


def test_key_above_key_bits_in_a_tiny_segment_is_reported(rs):
    import torch

    sizes = [100, 20_000, 40]
    n = sum(sizes)
    keys = synth.u32(n, 93, 0) >> np.uint32(20)  # 12-bit keys
    keys[20_120] = 1 << 12  # inside the last (warp) segment
    kd = to_dev(keys)
    off = to_dev(synth.segment_offsets(sizes))
    ws = rs.workspace(rs.rs_segmented_workspace_bytes(4, 0, n, 3, 12))
    out = torch.empty_like(kd)
    assert rs.rs_sort_segmented_u32(kd, out, None, None, off, 3, n, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE
