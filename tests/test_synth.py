"""The seeded input generator: pinned to SplitMix64's published outputs, the
device (torch) form equal to the numpy form bit for bit, and the
distributions with the shapes they claim."""
import os

import numpy as np
import pytest

import synth


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(x, 16) for x in (ln.strip() for ln in f) if x and not x.startswith("#")]


def test_splitmix64_published_outputs():
    """SplitMix64 seeded with state 0 (tests/golden/splitmix64_state0.txt).
    Seed 0 of dist 0, stream 0 has base mix(0) = 0, so its draws are that
    sequence."""
    assert int(synth.stream_base(0, 0, 0)) == 0
    want = read_golden("splitmix64_state0.txt")
    assert [int(v) for v in synth.u64(len(want), 0, 0, 0)] == want


@pytest.mark.parametrize("seed,dist,stream", [(0, 0, 0), (5, 20, 0), (3, 6, 11), (2**40 + 7, 9, 3)])
def test_torch_form_equals_numpy_form(seed, dist, stream):
    n = 50_001
    a = synth.u64(n, seed, dist, stream)
    b = synth.u64_torch(n, seed, dist, stream, chunk=4099).numpy().view(np.uint64)
    assert np.array_equal(a, b)
    a32 = synth.u32(n, seed, dist, stream)
    b32 = synth.u32_torch(n, seed, dist, stream, chunk=10_000).numpy().view(np.uint32)
    assert np.array_equal(a32, b32)


def test_distribution_shapes():
    n = 200_000
    assert synth.keys_u32(n, 1).max() < 1000
    s = synth.keys_u32(n, 3)
    assert np.all(s[1:] >= s[:-1]) and s[-1] > 2**32 - 2**32 // 1000
    assert np.array_equal(synth.keys_u32(n, 4), s[::-1])
    near = synth.keys_u32(n, 5)
    assert 0 < np.count_nonzero(near != s) <= 2 * (n // 100)
    g = synth.keys_u32(n, 6).astype(np.float64)
    assert abs(g.mean() - 2**31) < 0.02 * 2**20 and abs(g.std() - 2**20) < 0.03 * 2**20
    u = synth.keys_u32(n, 0).astype(np.float64)
    assert abs(u.mean() / 2**32 - 0.5) < 0.01


def test_log_uniform_sizes():
    sz = synth.log_uniform_sizes(20_000, 256, 2_000_000, seed=0)
    assert sz.min() >= 256 and sz.max() <= 2_000_000
    # the mean of a log-uniform law on [a, b] is (b - a) / ln(b / a)
    want = (2_000_000 - 256) / np.log(2_000_000 / 256)
    assert abs(sz.mean() / want - 1) < 0.03


@pytest.mark.parametrize("dist", [0, 1, 2, 3, 4, 5, 6])
def test_device_form_of_the_distributions_equals_numpy_form(dist):
    """keys_u32_torch / keys_u64_shaped_torch (the benchmark builds its large
    inputs with them on the GPU) give the numpy forms' bits; run here on the
    CPU device."""
    n = 30_011
    a = synth.keys_u32(n, dist, seed=3)
    b = synth.keys_u32_torch(n, dist, seed=3, chunk=7_001).numpy().view(np.uint32)
    assert np.array_equal(a, b)
    a64 = synth.keys_u64_shaped(n, dist, seed=4)
    b64 = synth.keys_u64_shaped_torch(n, dist, seed=4).numpy().view(np.uint64)
    assert np.array_equal(a64, b64)
