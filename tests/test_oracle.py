"""Pins for the CPU oracle, against facts the paper and the mathematics fix
rather than against the oracle's own formulas:

* sorted output is unique (Sec. 2: a nondecreasing permutation), so keys-only
  results must equal Python's ``sorted`` / numpy's sort;
* a stable sort (Sec. 2) of (key, index) pairs is unique too, so key-value
  results must equal a stable library sort;
* a single counting-sort pass (Algorithm 3) is a stable sort on one digit;
* after p passes, LSD radix (Algorithm 4) has sorted the keys stably on their
  low p*D bits (a most-significant-first order would fail this);
* the printed backward form of Algorithm 3 and the forward form agree;
* the bucket function (Sec. 2.3) is monotone, covers [0, nb), sends min to 0,
  and reduces to closed forms when nb divides the range or the range is 2^64.
"""
import itertools

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng(seed):
    return np.random.default_rng(seed)


def _stable_ref(keys, vals):
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


# ---------------------------------------------------------------- counting sort
@pytest.mark.parametrize("digit_bits,shift", [(1, 0), (4, 4), (8, 0), (8, 24), (11, 5), (16, 16)])
def test_counting_pass_is_stable_sort_on_one_digit(oracle, digit_bits, shift):
    keys = synth.u32(20000, 1, 0)
    vals = np.arange(keys.size, dtype=np.uint32)
    ok, ov = oracle.counting_pass(keys, vals, shift, digit_bits)
    digit = (keys.astype(np.uint64) >> np.uint64(shift)) & np.uint64((1 << digit_bits) - 1)
    order = np.argsort(digit, kind="stable")
    assert np.array_equal(ok, keys[order])
    assert np.array_equal(ov, vals[order])


@pytest.mark.parametrize("digit_bits", [1, 3, 8, 13])
def test_counting_pass_printed_backward_form_agrees(oracle, digit_bits):
    keys = synth.u32(5000, 2, 1) >> np.uint32(20)  # many ties
    vals = np.arange(keys.size, dtype=np.uint32)
    f = oracle.counting_pass(keys, vals, 2, digit_bits, backward=False)
    b = oracle.counting_pass(keys, vals, 2, digit_bits, backward=True)
    assert np.array_equal(f[0], b[0]) and np.array_equal(f[1], b[1])


def test_digit_counts_match_bincount(oracle):
    keys = synth.u32(30000, 3, 0)
    c = oracle.digit_counts(keys, 32, 8)
    assert c.shape == (4, 256)
    for p in range(4):
        d = (keys >> np.uint32(8 * p)) & np.uint32(255)
        assert np.array_equal(c[p], np.bincount(d, minlength=256))
    c7 = oracle.digit_counts(keys >> np.uint32(1), 31, 7)  # 5 passes, last holds 3 bits
    assert c7.shape == (5, 128) and int(c7[4, 8:].sum()) == 0
    assert all(int(c7[p].sum()) == keys.size for p in range(5))


# ---------------------------------------------------------------- radix sort
def test_radix_tiny_exhaustive(oracle):
    """Every sequence of length <= 5 over {0,1,2,3}, keys only and with the
    input index as value, against Python's stable ``sorted``."""
    for n in range(0, 6):
        for seq in itertools.product(range(4), repeat=n):
            keys = np.array(seq, dtype=np.uint32)
            vals = np.arange(n, dtype=np.uint32)
            want = sorted(zip(seq, range(n)), key=lambda kv: kv[0])
            ok, ov = oracle.radix_sort(keys, vals, key_bits=2, digit_bits=1)
            assert [int(x) for x in ok] == [k for k, _ in want]
            assert [int(x) for x in ov] == [v for _, v in want]


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 100_000])
@pytest.mark.parametrize("dist", [0, 1, 3, 4, 5, 6, 8])
def test_radix_u32_vs_numpy(oracle, n, dist):
    keys = synth.keys_u32(n, dist, seed=n)
    vals = synth.index_values(n)
    ok, ov = oracle.radix_sort(keys, vals, 32, 8)
    rk, rv = _stable_ref(keys, vals)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
    assert np.array_equal(oracle.radix_sort(keys, None, 32, 8), np.sort(keys))


@pytest.mark.parametrize("key_bits", [1, 7, 33, 40, 63, 64])
def test_radix_u64_vs_numpy(oracle, key_bits):
    keys = synth.keys_u64(20000, key_bits, seed=key_bits)
    vals = synth.index_values(keys.size)
    ok, ov = oracle.radix_sort(keys, vals, key_bits, 8)
    rk, rv = _stable_ref(keys, vals)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


def test_radix_every_digit_width_gives_the_same_result(oracle):
    keys = synth.keys_u32(30011, 6, seed=4)
    vals = synth.index_values(keys.size)
    ref = oracle.radix_sort(keys, vals, 32, 8)
    for D in range(1, 17):
        got = oracle.radix_sort(keys, vals, 32, D)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), D


@pytest.mark.parametrize("D", [3, 8])
def test_radix_partial_passes_sort_low_digits_first(oracle, D):
    keys = synth.u32(20000, 9, 0)
    vals = synth.index_values(keys.size)
    for p in range(1, oracle.num_passes(32, D) + 1):
        ok, ov = oracle.radix_sort(keys, vals, 32, D, max_passes=p)
        low = keys.astype(np.uint64) & np.uint64((1 << min(64, p * D)) - 1)
        order = np.argsort(low, kind="stable")
        assert np.array_equal(ok, keys[order]) and np.array_equal(ov, vals[order]), p


def test_radix_invariants(oracle):
    keys = synth.keys_u32(50000, 8, seed=1)
    out = oracle.radix_sort(keys)
    assert np.all(out[1:] >= out[:-1])                                    # nondecreasing
    u1, c1 = np.unique(keys, return_counts=True)
    u2, c2 = np.unique(out, return_counts=True)
    assert np.array_equal(u1, u2) and np.array_equal(c1, c2)              # permutation
    assert np.array_equal(oracle.radix_sort(out), out)                    # sorted input unchanged
    vals = synth.index_values(keys.size)
    ok, ov = oracle.radix_sort(keys, vals)
    same = ok[1:] == ok[:-1]
    assert np.all(ov[1:][same] > ov[:-1][same])                           # stable


def test_radix_rejects_keys_above_key_bits(oracle):
    with pytest.raises(oracle.OracleError):
        oracle.radix_sort(np.array([0, 300], np.uint32), None, 8, 8)


def test_radix_degenerate(oracle):
    e = np.empty(0, np.uint32)
    assert oracle.radix_sort(e).size == 0
    one = np.array([7], np.uint32)
    assert np.array_equal(oracle.radix_sort(one), one)
    same = np.full(1000, 0xFFFFFFFF, np.uint32)
    vals = synth.index_values(1000)
    ok, ov = oracle.radix_sort(same, vals)
    assert np.array_equal(ok, same) and np.array_equal(ov, vals)


# ---------------------------------------------------------------- bucket function
def test_bucket_index_closed_form_when_nb_divides_range(oracle):
    # R = 2^31, nb = 2^16: every bucket holds exactly R/nb consecutive keys
    R, nb = 2**31, 2**16
    width = R // nb
    for k in [0, 1, width - 1, width, width + 1, R - 1, 123456789]:
        assert oracle.bucket_index(k, 0, R - 1, nb) == k // width
    # shifted range
    assert oracle.bucket_index(1000 + 3 * 7 + 6, 1000, 1000 + 7 * 10 - 1, 10) == 3


def test_bucket_index_full_u64_range_is_a_high_product(oracle):
    # R = 2^64: floor(k * nb / 2^64) is the high 64 bits of the 128-bit product
    rng = _rng(7)
    for _ in range(200):
        k = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        nb = int(rng.integers(1, 2**40))
        assert oracle.bucket_index(k, 0, 2**64 - 1, nb) == (k * nb) >> 64
    assert oracle.bucket_index(2**64 - 1, 0, 2**64 - 1, 2**63) == 2**63 - 1


@pytest.mark.parametrize("lo,hi,nb", [(0, 999, 62500), (0, 2**31 - 1, 62500), (5, 5, 3),
                                      (0, 2**32 - 1, 6_250_000), (17, 10**6, 999), (0, 10, 1)])
def test_bucket_index_properties(oracle, lo, hi, nb):
    R = hi - lo + 1
    ks = sorted({lo, hi, lo + 1 if hi > lo else lo, (lo + hi) // 2, hi - 1 if hi > lo else hi}
                | set(int(x) for x in _rng(lo + nb).integers(lo, hi + 1, 300)))
    ids = [oracle.bucket_index(k, lo, hi, nb) for k in ks]
    assert all(0 <= b < nb for b in ids)
    assert all(a <= b for a, b in zip(ids, ids[1:]))                  # monotone in k
    assert oracle.bucket_index(lo, lo, hi, nb) == 0
    if nb <= R:
        assert oracle.bucket_index(hi, lo, hi, nb) == nb - 1
    else:
        assert oracle.bucket_index(hi, lo, hi, nb) <= nb - 1


def test_bucket_sizes_over_a_full_range_are_floor_or_ceil(oracle):
    # every key of [lo, hi] once: each bucket receives floor(R/nb) or ceil(R/nb) keys
    lo, hi = 3, 3 + 9999
    keys = np.arange(lo, hi + 1, dtype=np.uint32)
    for nb in [1, 7, 10, 333, 10000]:
        c = oracle.bucket_counts(keys, lo, hi, nb)
        R = hi - lo + 1
        assert int(c.sum()) == R
        assert set(int(x) for x in np.unique(c)) <= {R // nb, -(-R // nb)}


# ---------------------------------------------------------------- bucket sort
@pytest.mark.parametrize("dist", [0, 1, 3, 4, 5, 6, 7, 8])
def test_bucket_sort_equals_stable_sort(oracle, dist):
    n = 20000
    keys = synth.keys_u32(n, dist, seed=dist)
    vals = synth.index_values(n)
    lo, hi = synth.DECLARED_BOUNDS[dist]
    ok, ov = oracle.bucket_sort(keys, vals, lo, hi, max(1, n // 16))
    rk, rv = _stable_ref(keys, vals)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
    rr = oracle.radix_sort(keys, vals)
    assert np.array_equal(ok, rr[0]) and np.array_equal(ov, rr[1])


@pytest.mark.parametrize("nb", [1, 2, 5000, 20000, 10**6])
def test_bucket_sort_bucket_counts_edge(oracle, nb):
    keys = synth.keys_u32(5000, 0, seed=3) >> np.uint32(16)
    vals = synth.index_values(keys.size)
    ok, ov = oracle.bucket_sort(keys, vals, 0, 65535, nb)
    rk, rv = _stable_ref(keys, vals)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)


def test_bucket_sort_u64_and_computed_bounds(oracle):
    keys = synth.keys_u64(10000, 64, seed=5)
    vals = synth.index_values(keys.size)
    ok, ov = oracle.bucket_sort(keys, vals)  # bounds from the data, nb = n // 16
    rk, rv = _stable_ref(keys, vals)
    assert np.array_equal(ok, rk) and np.array_equal(ov, rv)
    c = oracle.bucket_counts(keys, int(keys.min()), int(keys.max()), 625)
    assert int(c.sum()) == keys.size


def test_bucket_sort_min_equals_max_and_out_of_range(oracle):
    keys = np.full(100, 42, np.uint32)
    assert np.array_equal(oracle.bucket_sort(keys, None, 42, 42, 7), keys)
    with pytest.raises(oracle.OracleError):
        oracle.bucket_sort(np.array([1, 50], np.uint32), None, 0, 10, 4)


def test_minmax(oracle):
    keys = synth.keys_u32(777, 6, seed=2)
    assert oracle.minmax(keys) == (int(keys.min()), int(keys.max()))


def test_segmented_oracle_matches_per_segment_sort(oracle):
    sizes = [0, 1, 5, 300, 0, 1000]
    off = synth.segment_offsets(sizes)
    keys = synth.u32(int(off[-1]), 11, 0)
    vals = synth.index_values(keys.size)
    ok, ov = oracle.segmented_radix_sort(keys, off, vals)
    for s in range(len(sizes)):
        a, b = int(off[s]), int(off[s + 1])
        rk, rv = _stable_ref(keys[a:b], vals[a:b])
        assert np.array_equal(ok[a:b], rk) and np.array_equal(ov[a:b], rv)


# ---------------------------------------------------------------- typed keys
def test_typed_signed_matches_numpy_stable_sort(oracle):
    rng = np.random.default_rng(5)
    for dt, lo, hi in [(np.int32, -2**31, 2**31), (np.int64, -2**63, 2**63 - 1)]:
        x = rng.integers(lo, hi, 20_000, dtype=dt)
        x[:6] = [np.iinfo(dt).min, np.iinfo(dt).max, -1, 0, 1, np.iinfo(dt).min]
        x[100:200] = x[300:400]  # duplicates
        order = np.argsort(x, kind="stable")
        k, v = oracle.sort_typed(x, np.arange(x.size, dtype=np.uint32))
        assert np.array_equal(k, x[order]) and np.array_equal(v, order.astype(np.uint32))


def test_typed_float_matches_numpy_without_nan_and_negative_zero(oracle):
    rng = np.random.default_rng(6)
    for dt in (np.float32, np.float64):
        x = (rng.standard_normal(20_000) * 10.0 ** rng.integers(-30, 30, 20_000)).astype(dt)
        x[:4] = [np.inf, -np.inf, np.finfo(dt).tiny, -np.finfo(dt).max]
        x[1000:1100] = x[2000:2100]
        x[x == 0] = 1  # numpy treats -0 and +0 as equal; totalOrder does not
        order = np.argsort(x, kind="stable")
        k, v = oracle.sort_typed(x, np.arange(x.size, dtype=np.uint32))
        assert np.array_equal(k.view(np.uint8), x[order].view(np.uint8))
        assert np.array_equal(v, order.astype(np.uint32))


def test_typed_float_total_order_of_special_values(oracle):
    """IEEE 754-2008 totalOrder: -NaN < -inf < -1 < -denormal < -0 < +0 <
    +denormal < 1 < +inf < +NaN."""
    for dt, ut in ((np.float32, np.uint32), (np.float64, np.uint64)):
        qnan = np.array([np.nan], dt).view(ut)[0]
        sign = ut(1) << ut(8 * np.dtype(dt).itemsize - 1)
        want_bits = [qnan | sign] + [np.array([v], dt).view(ut)[0] for v in
                                     (-np.inf, -1.0, -np.finfo(dt).smallest_subnormal, -0.0, 0.0,
                                      np.finfo(dt).smallest_subnormal, 1.0, np.inf)] + [qnan]
        want = np.array(want_bits, ut)
        perm = np.array([9, 3, 0, 7, 5, 1, 8, 2, 6, 4])
        got = oracle.sort_typed(want[perm].view(dt)).view(ut)
        assert np.array_equal(got, want)


def test_typed_float32_total_order_golden(oracle):
    """The IEEE-754 totalOrder sequence of tests/golden/ieee754_total_order.txt,
    shuffled, comes back in order; reversed for descending."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ieee754_total_order.txt")
    with open(path) as f:
        want = np.array([int(x, 16) for x in (ln.strip() for ln in f) if x and not x.startswith("#")], np.uint32)
    perm = np.array([3, 9, 0, 6, 1, 8, 4, 2, 7, 5])
    assert np.array_equal(oracle.sort_typed(want[perm].view(np.float32)).view(np.uint32), want)
    assert np.array_equal(oracle.sort_typed(want[perm].view(np.float32), descending=True).view(np.uint32),
                          want[::-1])


def test_typed_descending_is_the_stable_reverse_order(oracle):
    rng = np.random.default_rng(7)
    x = rng.integers(-50, 50, 5000, dtype=np.int32)
    k, v = oracle.sort_typed(x, np.arange(x.size, dtype=np.uint32), descending=True)
    order = sorted(range(x.size), key=lambda i: (-int(x[i]), i))
    assert np.array_equal(v, np.array(order, np.uint32)) and np.array_equal(k, x[order])
    f = rng.standard_normal(3000).astype(np.float64)
    f[::7] = f[3]
    kf, vf = oracle.sort_typed(f, np.arange(f.size, dtype=np.uint32), descending=True)
    order = sorted(range(f.size), key=lambda i: (-float(f[i]), i))
    assert np.array_equal(vf, np.array(order, np.uint32))


def test_typed_tiny_exhaustive_against_sorted(oracle):
    alphabet = np.array([-2, -1, 0, 3], np.int32)
    import itertools
    for n in range(0, 5):
        for combo in itertools.product(range(4), repeat=n):
            x = alphabet[list(combo)] if n else np.zeros(0, np.int32)
            for desc in (False, True):
                k, v = oracle.sort_typed(x, np.arange(n, dtype=np.uint32), descending=desc)
                order = sorted(range(n), key=lambda i: ((-1 if desc else 1) * int(x[i]), i))
                assert list(v) == order


def test_typed_unsigned_equals_radix(oracle):
    x = synth.u32(10_000, 8, 0)
    assert np.array_equal(oracle.sort_typed(x), oracle.radix_sort(x, None, 32))
