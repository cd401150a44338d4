"""GPU parity of the LSD radix path against the CPU oracle, element by
element, zero tolerance (integer work is bit-exact).  Every call goes through
the C ABI via the ctypes binding."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _sort_dev(rs, keys_np, vals_np=None, key_bits=0, cfg=None, in_place=False):
    import torch

    k = to_dev(keys_np)
    v = to_dev(vals_np) if vals_np is not None else None
    if in_place:
        out, outv = rs.sort(k, v, key_bits, out=k, out_values=v, config=cfg)
    else:
        out, outv = rs.sort(k, v, key_bits, config=cfg)
    torch.cuda.synchronize()
    ko = from_dev(out, keys_np.dtype)
    vo = from_dev(outv, np.uint32) if vals_np is not None else None
    return ko, vo


def _check(rs, oracle, keys, vals=None, key_bits=0, cfg=None, in_place=False, what=""):
    kbits = key_bits or 8 * keys.dtype.itemsize
    got_k, got_v = _sort_dev(rs, keys, vals, key_bits, cfg, in_place)
    if vals is None:
        want = oracle.radix_sort(keys, None, kbits, 8)
        assert_same(got_k, want, what)
    else:
        wk, wv = oracle.radix_sort(keys, vals, kbits, 8)
        assert_same(got_k, wk, what + " keys")
        assert_same(got_v, wv, what + " values")


def test_small_config_1m_uniform_31bit(rs, oracle):
    """1,000,000 u32 keys uniform in [0, 2^31), seed 0: 8-bit digits, 4 passes."""
    keys = synth.u32(1_000_000, 0, 0) >> np.uint32(1)
    _check(rs, oracle, keys, None, 32, what="1M uniform")
    _check(rs, oracle, keys, None, 31, what="1M uniform key_bits=31")


# around the single-block limit (4096 keys) and the u32 scatter tiles (6144 keys
# keys-only, 3072 with values; 4608 for the 256x18 shape)
TILE_SIZES = [0, 1, 2, 3, 31, 33, 3840, 4095, 4096, 4097, 4607, 4608, 4609, 6143, 6144, 6145, 2 * 6144 + 7,
              65537, (1 << 20) + 3]


@pytest.mark.parametrize("n", TILE_SIZES)
def test_sizes_u32(rs, oracle, n):
    keys = synth.u32(n, 100 + n % 97, 0)
    _check(rs, oracle, keys, None, what=f"u32 n={n}")
    _check(rs, oracle, keys, synth.index_values(n), what=f"u32 kv n={n}")


@pytest.mark.parametrize("n", [0, 1, 5, 3071, 4096, 4097, 6143, 6144, 6145, 2560 * 3 + 1, 100_003])
def test_sizes_u64(rs, oracle, n):
    keys = synth.keys_u64(n, 64, seed=n)
    _check(rs, oracle, keys, None, what=f"u64 n={n}")
    _check(rs, oracle, keys, synth.index_values(n), what=f"u64 kv n={n}")


@pytest.mark.parametrize("dist", list(synth.DISTS))
def test_distributions_u32(rs, oracle, dist):
    n = 300_007
    keys = synth.keys_u32(n, dist, seed=1)
    _check(rs, oracle, keys, None, what=synth.DISTS[dist])
    _check(rs, oracle, keys, synth.index_values(n), what=synth.DISTS[dist] + " kv")


@pytest.mark.parametrize("key_bits", [1, 4, 7, 8, 9, 16, 17, 31, 32])
def test_key_bits_u32(rs, oracle, key_bits):
    n = 50_000
    keys = synth.u32(n, key_bits, 0) >> np.uint32(32 - key_bits)
    _check(rs, oracle, keys, synth.index_values(n), key_bits, what=f"key_bits={key_bits}")


@pytest.mark.parametrize("key_bits", [1, 33, 40, 57, 63, 64])
def test_key_bits_u64(rs, oracle, key_bits):
    n = 40_000
    keys = synth.keys_u64(n, key_bits, seed=key_bits)
    _check(rs, oracle, keys, synth.index_values(n), key_bits, what=f"u64 key_bits={key_bits}")


def test_every_compiled_config_gives_identical_bits(rs, oracle):
    n = 200_003
    for kb in (4, 8):
        for has_v in (False, True):
            keys = synth.u32(n, 7, 0) if kb == 4 else synth.keys_u64(n, 64, seed=7)
            vals = synth.index_values(n) if has_v else None
            for i in range(rs.rs_config_count(kb, has_v)):
                cfg = rs.rs_config_get(kb, has_v, i)
                _check(rs, oracle, keys, vals, 0, cfg.as_tuple(), what=f"cfg {cfg.as_tuple()} kb={kb} v={has_v}")


@pytest.mark.parametrize("key_bits", [32, 24])  # 4 passes (even), 3 passes (odd)
def test_in_place(rs, oracle, key_bits):
    n = 123_457
    keys = synth.u32(n, 3, 0) >> np.uint32(32 - key_bits)
    _check(rs, oracle, keys, synth.index_values(n), key_bits, in_place=True, what=f"in place {key_bits}")


def test_misaligned_pointers(rs, oracle):
    import torch

    n = 77_777
    keys = synth.u32(n + 3, 4, 0)
    vals = synth.index_values(n + 3)
    kd, vd = to_dev(keys), to_dev(vals)
    out = torch.empty(n + 3, dtype=torch.int32, device="cuda")
    outv = torch.empty(n + 3, dtype=torch.int32, device="cuda")
    for off in (1, 2, 3):  # 4, 8, 12 bytes past a 16-byte boundary
        nb = rs.rs_workspace_bytes(0, 4, 1, n, 32, 0, 0)
        ws = rs.workspace(nb)
        rc = rs.rs_sort_u32(kd[off:off + n], out[off:off + n], vd[off:off + n], outv[off:off + n], n, 32, ws,
                            ws.numel())
        assert rc == 0
        torch.cuda.synchronize()
        wk, wv = oracle.radix_sort(keys[off:off + n], vals[off:off + n])
        assert_same(from_dev(out[off:off + n], np.uint32), wk, f"misaligned keys {off}")
        assert_same(from_dev(outv[off:off + n], np.uint32), wv, f"misaligned values {off}")


def test_all_equal_and_extreme_keys(rs, oracle):
    for fill in (0, 0xFFFFFFFF, 0x80000000):
        keys = np.full(50_001, fill, np.uint32)
        _check(rs, oracle, keys, synth.index_values(keys.size), what=f"all {fill:#x}")
    keys = np.array([0xFFFFFFFF, 0, 0xFFFFFFFF, 1, 0] * 1000, np.uint32)
    _check(rs, oracle, keys, synth.index_values(keys.size), what="extremes")
    k64 = np.array([2**64 - 1, 0, 2**63, 2**63 - 1] * 2000, np.uint64)
    _check(rs, oracle, k64, synth.index_values(k64.size), what="u64 extremes")


def test_digit_counts_match_oracle(rs, oracle):
    keys = synth.keys_u32(500_001, 6, seed=2)
    for D in (4, 8, 11):
        got = rs.digit_counts(to_dev(keys), 32, D).cpu().numpy()
        want = oracle.digit_counts(keys, 32, D).astype(np.int64)
        assert_same(got, want, f"digit counts D={D}")
    k64 = synth.keys_u64(100_000, 40, seed=3)
    got = rs.digit_counts(to_dev(k64), 40, 8).cpu().numpy()
    assert_same(got, oracle.digit_counts(k64, 40, 8).astype(np.int64), "u64 digit counts")


@pytest.mark.parametrize("shift,D", [(0, 8), (8, 8), (24, 8), (3, 11), (28, 4), (21, 11)])
def test_single_counting_pass_matches_oracle(rs, oracle, shift, D):
    n = 250_013
    keys = synth.u32(n, shift + D, 0)
    vals = synth.index_values(n)
    ok, ov = rs.counting_pass(to_dev(keys), to_dev(vals), shift, D)
    wk, wv = oracle.counting_pass(keys, vals, shift, D)
    assert_same(from_dev(ok, np.uint32), wk, "pass keys")
    assert_same(from_dev(ov, np.uint32), wv, "pass values")
    k64 = synth.keys_u64(n, 64, seed=shift)
    ok, ov = rs.counting_pass(to_dev(k64), to_dev(vals), shift + 32, D)
    wk, wv = oracle.counting_pass(k64, vals, shift + 32, D)
    assert_same(from_dev(ok, np.uint64), wk, "u64 pass keys")
    assert_same(from_dev(ov, np.uint32), wv, "u64 pass values")


def test_key_above_key_bits_is_reported(rs):
    import torch

    keys = synth.u32(100_000, 5, 0) >> np.uint32(20)  # 12-bit keys
    keys[777] = 1 << 12
    kd = to_dev(keys)
    nb = rs.rs_workspace_bytes(0, 4, 0, keys.size, 12, 0, 0)
    ws = rs.workspace(nb)
    out = torch.empty_like(kd)
    assert rs.rs_sort_u32(kd, out, None, None, keys.size, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE
    assert rs.get_status(ws) == 0  # cleared by the read
    # the same workspace keeps working
    keys[777] = 5
    kd = to_dev(keys)
    assert rs.rs_sort_u32(kd, out, None, None, keys.size, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 0
    assert np.array_equal(from_dev(out, np.uint32), np.sort(keys))


@pytest.mark.parametrize("kb,with_values", [(4, False), (4, True), (8, False), (8, True)])
def test_small_array_is_one_block_sort(rs, oracle, kb, with_values):
    """Arrays of at most 4096 keys are sorted by one shared-memory block: one
    kernel launch, the same bits as the oracle, in place too."""
    import torch

    n = 4000
    keys = synth.u32(n, 61, 0) if kb == 4 else synth.keys_u64(n, 64, seed=61)
    vals = synth.index_values(n) if with_values else None
    kd = to_dev(keys)
    vd = to_dev(vals) if with_values else None
    torch.cuda.synchronize()
    before = rs.rs_launch_count()
    ok, ov = rs.sort(kd, vd)
    torch.cuda.synchronize()
    assert rs.rs_launch_count() - before == 1
    if with_values:
        wk, wv = oracle.radix_sort(keys, vals, 8 * kb)
        assert_same(from_dev(ov, np.uint32), wv, "small values")
    else:
        wk = oracle.radix_sort(keys, None, 8 * kb)
    assert_same(from_dev(ok, keys.dtype), wk, "small keys")
    ok2, ov2 = rs.sort(kd, vd, out=kd, out_values=vd)
    torch.cuda.synchronize()
    assert_same(from_dev(kd, keys.dtype), wk, "small in place")


def test_small_key_above_key_bits_is_reported(rs):
    import torch

    keys = synth.u32(1000, 62, 0) >> np.uint32(20)  # 12-bit keys
    keys[500] = 1 << 12
    kd = to_dev(keys)
    ws = rs.workspace(rs.rs_workspace_bytes(0, 4, 0, keys.size, 12, 0, 0))
    out = torch.empty_like(kd)
    assert rs.rs_sort_u32(kd, out, None, None, keys.size, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 3  # RS_ERR_KEY_RANGE
    keys[500] = 7
    assert rs.rs_sort_u32(to_dev(keys), out, None, None, keys.size, 12, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 0
    assert np.array_equal(from_dev(out, np.uint32), np.sort(keys))


def test_bounded_wait_reports_timeout_and_context_survives(rs, oracle):
    """A tile that never publishes makes later tiles give up after a short
    bounded wait; the call completes, reports RS_ERR_DEVICE_TIMEOUT, and the
    context stays usable."""
    import torch

    n = 20 * 3840
    keys = synth.u32(n, 9, 0)
    kd = to_dev(keys)
    out = torch.empty_like(kd)
    ws = rs.workspace(rs.rs_workspace_bytes(0, 4, 0, n, 32, 0, 0))
    try:
        rs.rs_set_debug(2000, 5)
        assert rs.rs_sort_u32(kd, out, None, None, n, 32, ws, ws.numel()) == 0
        assert rs.get_status(ws) == 6  # RS_ERR_DEVICE_TIMEOUT
    finally:
        rs.rs_set_debug(0, -1)
    assert rs.rs_sort_u32(kd, out, None, None, n, 32, ws, ws.numel()) == 0
    assert rs.get_status(ws) == 0
    assert_same(from_dev(out, np.uint32), oracle.radix_sort(keys), "after timeout")


@pytest.mark.slow
def test_full_size_100m_u32_uniform(rs, oracle):
    """The 100M-key u32 uniform workload the benchmark times, checked in full."""
    keys = synth.keys_u32(100_000_000, 0, seed=0)
    _check(rs, oracle, keys, None, 32, what="100M u32")


@pytest.mark.slow
def test_full_size_100m_u64_kv(rs, oracle):
    """100M u64 keys uniform in [0, 2^64) with index values: 8 passes."""
    import torch

    n = 100_000_000
    keys = synth.keys_u64(n, 64, seed=0)
    vals = synth.index_values(n)
    gk, gv = _sort_dev(rs, keys, vals, 64)
    torch.cuda.empty_cache()
    wk, wv = oracle.radix_sort(keys, vals, 64, 8)
    assert_same(gk, wk, "100M u64 keys")
    assert_same(gv, wv, "100M u64 values")


@pytest.mark.slow
def test_full_size_50m_u64_40bit_trimmed(rs, oracle):
    keys = synth.keys_u64(50_000_000, 40, seed=0)
    _check(rs, oracle, keys, None, 40, what="50M u64 40-bit")
