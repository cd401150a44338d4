"""Host-side arithmetic of the benchmark: the algorithmic bytes that the
roofline divides by the kernel time, pinned to the figures worked out for
each workload (one counting read of the keys, then one read and one write of
keys and values per pass)."""
import pytest


def test_radix_bytes_per_key():
    import bench

    n = 10**8
    # u32 keys only, 8-bit digits: 4 + 4 passes x 8 = 36 B/key -> 3.6 GB
    assert bench.sort_bytes("radix", n, 4, False) == 36 * n
    # u64 keys + u32 values, 8 passes: 8 + 8 x 24 = 200 B/key -> 20 GB
    assert bench.sort_bytes("radix", n, 8, True) == 200 * n
    # u64 keys below 2^40: 5 passes at 8-bit digits (88 B/key), 4 at 10-bit (72)
    assert bench.sort_bytes("radix", n, 8, False, key_bits=40) == 88 * n
    assert bench.sort_bytes("radix", n, 8, False, key_bits=40, digit_bits=10) == 72 * n
    # trimming to key_bits: 20-bit keys in 3 passes of 8 bits
    assert bench.sort_bytes("radix", n, 4, False, key_bits=20) == (4 + 3 * 8) * n


def test_pass_and_bucket_bytes():
    import bench

    n = 10**8
    # one scatter pass of 100M u32 keys: 800 MB (the roofline's per-launch figure)
    assert bench.pass_bytes(n, 4, False) == 8 * 10**8
    assert bench.pass_bytes(n, 8, True) == 24 * n
    # bucket sort, u32 keys only: 4 + 8 + 8 = 20 B/key -> 2.0 GB
    assert bench.sort_bytes("bucket", n, 4, False) == 20 * n
    assert bench.sort_bytes("bucket", n, 8, True) == (8 + 2 * 24) * n


@pytest.mark.parametrize("kind,per_key", [(0, 36), (1, 200)])
def test_served_request_bytes(kind, per_key):
    import bench

    assert bench.served_bytes(1000, kind) == per_key * 1000
