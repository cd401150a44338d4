"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 3.1) and the
benchmark configurations.  Shared by the tests, the smoke check and the
benchmark; it holds no sorting arithmetic.

Random numbers come from one counter-based generator: output i of stream s is
SplitMix64's mixing function applied to base(s) + (i + 1) * gamma, where gamma
is SplitMix64's odd increment (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  The stream base is itself the
mix of (seed XOR (dist_id << 32) XOR (stream << 48)).  Everything is integer
arithmetic modulo 2^64 in numpy, so x86 and arm64 produce identical bytes.

Uniform integers in [0, R) use Lemire's multiply-shift (2019, "Fast random
integer generation in an interval") without the rejection step: a 32-bit draw
u maps to (u * R) >> 32.  The bias is below R / 2^32 and does not matter for
synthetic sort inputs.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 24

# Distribution ids.  0-6 are the seven distributions of the 100M-key u32
# workload; 7-9 reproduce the shapes of the paper's input cases 3, 6 and 5.
DISTS = {
    0: "uniform_u32",          # uniform over [0, 2^32) (control)
    1: "uniform_small_1000",   # uniform over [0, 1000)
    2: "uniform_large_u32",    # uniform over [0, 2^32), a second stream
    3: "sorted",               # nondecreasing, spread over [0, 2^32)
    4: "reverse_sorted",       # dist 3 reversed
    5: "nearly_sorted",        # dist 3 with n // 100 random swaps
    6: "gaussian",             # mean 2^31, sd 2^20, clipped to [0, 2^32 - 1]
    7: "sorted_95",            # sorted over [0, 1e6), then 5% of slots overwritten
    8: "third_one_value",      # n // 3 copies of 500000, rest uniform over [0, 1e6)
    9: "uniform_1e8",          # uniform over [0, 1e8)
}
DIST_IDS = {v: k for k, v in DISTS.items()}
# Declared [min, max] of each distribution (the paper's "between 0 and M").
DECLARED_BOUNDS = {
    0: (0, 2**32 - 1), 1: (0, 999), 2: (0, 2**32 - 1), 3: (0, 2**32 - 1), 4: (0, 2**32 - 1),
    5: (0, 2**32 - 1), 6: (0, 2**32 - 1), 7: (0, 999_999), 8: (0, 999_999), 9: (0, 10**8 - 1),
}


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_base(seed: int, dist_id: int = 0, stream: int = 0) -> np.uint64:
    s = np.array([(seed ^ (dist_id << 32) ^ (stream << 48)) & (2**64 - 1)], np.uint64)
    return _mix(s)[0]


def u64(n: int, seed: int, dist_id: int = 0, stream: int = 0, start: int = 0) -> np.ndarray:
    """n raw 64-bit draws of one stream, counters start+1 .. start+n."""
    base = stream_base(seed, dist_id, stream)
    out = np.empty(n, np.uint64)
    with np.errstate(over="ignore"):
        for a in range(0, n, _CHUNK):
            b = min(n, a + _CHUNK)
            ctr = np.arange(start + a + 1, start + b + 1, dtype=np.uint64)
            out[a:b] = _mix(base + ctr * GAMMA)
    return out


def _signed(v: int) -> int:
    return v - (1 << 64) if v >= (1 << 63) else v


def u64_torch_range(a: int, b: int, seed: int, dist_id: int = 0, stream: int = 0, device="cpu"):
    """Draws a .. b-1 of u64() (counters a+1 .. b) as an int64 torch tensor
    on `device`, same bits: for inputs too large to build on the host.
    int64 multiplication wraps modulo 2^64 like uint64; right shifts are
    made logical by masking."""
    import torch

    base = _signed(int(stream_base(seed, dist_id, stream)))
    g, m1, m2 = _signed(int(GAMMA)), _signed(int(_M1)), _signed(int(_M2))

    def srl(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    z = torch.arange(a + 1, b + 1, dtype=torch.int64, device=device)
    z.mul_(g).add_(base)
    z = (z ^ srl(z, 30)) * m1
    z = (z ^ srl(z, 27)) * m2
    return z ^ srl(z, 31)


def u64_torch(n: int, seed: int, dist_id: int = 0, stream: int = 0, device="cpu", chunk: int = 1 << 27):
    """u64() as an int64 torch tensor on `device` (same bits)."""
    import torch

    out = torch.empty(n, dtype=torch.int64, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = u64_torch_range(a, b, seed, dist_id, stream, device)
    return out


def u32_torch(n: int, seed: int, dist_id: int = 0, stream: int = 0, device="cpu", chunk: int = 1 << 27):
    """u32() as an int32 torch tensor on `device` (same bits): the high
    halves, taken with an arithmetic shift so that the int32 cast is exact."""
    import torch

    out = torch.empty(n, dtype=torch.int32, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = (u64_torch_range(a, b, seed, dist_id, stream, device) >> 32).to(torch.int32)
    return out


def u32(n: int, seed: int, dist_id: int = 0, stream: int = 0) -> np.ndarray:
    """n 32-bit draws: the high halves of the 64-bit draws."""
    return (u64(n, seed, dist_id, stream) >> np.uint64(32)).astype(np.uint32)


def uniform_below(n: int, R: int, seed: int, dist_id: int, stream: int = 0) -> np.ndarray:
    """n integers in [0, R), R <= 2^32, by multiply-shift of 32-bit draws."""
    if R == 2**32:
        return u32(n, seed, dist_id, stream)
    d = u32(n, seed, dist_id, stream).astype(np.uint64)
    with np.errstate(over="ignore"):
        return ((d * np.uint64(R)) >> np.uint64(32)).astype(np.uint32)


def _sorted_spread(n: int, seed: int, dist_id: int, hi: int) -> np.ndarray:
    """A nondecreasing sequence over [0, hi) built without sorting: slot i holds
    floor(i * hi / n) plus a random offset below the slot width."""
    if n == 0:
        return np.empty(0, np.uint32)
    i = np.arange(n, dtype=np.uint64)
    width = max(1, hi // n)
    with np.errstate(over="ignore"):
        base = (i * np.uint64(hi)) // np.uint64(n)
        off = (u32(n, seed, dist_id, 1).astype(np.uint64) * np.uint64(width)) >> np.uint64(32)
    v = np.minimum(base + off, np.uint64(hi - 1))
    return v.astype(np.uint32)


def keys_u32(n: int, dist: int | str = 0, seed: int = 0) -> np.ndarray:
    """n uint32 keys of one of the distributions in DISTS."""
    dist_id = DIST_IDS[dist] if isinstance(dist, str) else int(dist)
    if dist_id in (0, 2):
        return u32(n, seed, dist_id)
    if dist_id == 1:
        return uniform_below(n, 1000, seed, dist_id)
    if dist_id == 3:
        return _sorted_spread(n, seed, 3, 2**32)
    if dist_id == 4:
        return _sorted_spread(n, seed, 3, 2**32)[::-1].copy()
    if dist_id == 5:
        a = _sorted_spread(n, seed, 3, 2**32)
        m = n // 100
        if m:
            # swap pairs (x_j, y_j) one after another, j = 0 .. m-1
            xs = uniform_below(m, n, seed, 5, 2).astype(np.int64)
            ys = uniform_below(m, n, seed, 5, 3).astype(np.int64)
            for x, y in zip(xs.tolist(), ys.tolist()):
                a[x], a[y] = a[y], a[x]
        return a
    if dist_id == 6:
        return gaussian_u32(n, seed)
    if dist_id == 7:
        a = _sorted_spread(n, seed, 7, 10**6)
        m = n // 20
        if m:
            pos = uniform_below(m, n, seed, 7, 2).astype(np.int64)
            a[pos] = uniform_below(m, 10**6, seed, 7, 3)
        return a
    if dist_id == 8:
        a = uniform_below(n, 10**6, seed, 8)
        m = n // 3
        if m:
            # put 500000 at the n // 3 distinct slots (step * j + start) mod n,
            # j < n // 3, with step coprime to n
            r = u64(2, seed, 8, 2)
            step = int(r[0] % np.uint64(n)) | 1
            while math.gcd(step, n) != 1:
                step += 2
            start = int(r[1] % np.uint64(n))
            pos = (np.arange(m, dtype=np.int64) * step + start) % n
            a[pos] = 500_000
        return a
    if dist_id == 9:
        return uniform_below(n, 10**8, seed, 9)
    raise ValueError(f"unknown distribution {dist}")


def gaussian_u32(n: int, seed: int = 0) -> np.ndarray:
    """Mean 2^31, sd 2^20: the Irwin-Hall sum S of twelve 32-bit uniforms has
    mean 6 * 2^32 and sd 2^32 (up to the discreteness of the draws), so
    2^31 + ((S - 6 * 2^32) >> 12) has sd 2^20.  Integer only, clipped."""
    out = np.empty(n, np.uint32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        m = b - a
        s = np.zeros(m, np.int64)
        for j in range(6):
            d = u64(m, seed, 6, 10 + j, start=a)
            s += (d >> np.uint64(32)).astype(np.int64)
            s += (d & np.uint64(0xFFFFFFFF)).astype(np.int64)
        v = (2**31) + ((s - 6 * 2**32) >> 12)
        out[a:b] = np.clip(v, 0, 2**32 - 1).astype(np.uint32)
    return out


# The paper's six input cases (Sec. 3.1): (description, M); keys lie in [0, M).
PAPER_CASES = {
    1: ("uniform, M = 10^6", 10**6),
    2: ("sorted, M = 10^6", 10**6),
    3: ("95% sorted, M = 10^6", 10**6),
    4: ("small range, M = 10^4", 10**4),
    5: ("large range, M = 10^8", 10**8),
    6: ("n/3 equal to one value, M = 10^6", 10**6),
}


def paper_case_keys(n: int, case: int, seed: int = 0) -> np.ndarray:
    """n uint32 keys shaped like the paper's input case (Sec. 3.1)."""
    if case == 1:
        return uniform_below(n, 10**6, seed, 61)
    if case == 2:
        return _sorted_spread(n, seed, 62, 10**6)
    if case == 3:
        return keys_u32(n, 7, seed)
    if case == 4:
        return uniform_below(n, 10**4, seed, 64)
    if case == 5:
        return keys_u32(n, 9, seed)
    if case == 6:
        return keys_u32(n, 8, seed)
    raise ValueError(f"no paper case {case}")


def _srl_t(z, k: int):
    """Logical right shift of an int64 torch tensor holding uint64 bits."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _hi32_t(n: int, seed: int, dist_id: int, stream: int, device, start: int = 0):
    """The 32-bit draws of u32() (counters start+1 .. start+n) as non-negative
    int64 values on `device`."""
    return _srl_t(u64_torch_range(start, start + n, seed, dist_id, stream, device), 32)


def _uniform_below_t(n: int, R: int, seed: int, dist_id: int, stream: int, device):
    """uniform_below() on `device` as int64 values (same numbers)."""
    d = _hi32_t(n, seed, dist_id, stream, device)
    return d if R == 2**32 else _srl_t(d * R, 32)


def _sorted_spread_t(n: int, seed: int, dist_id: int, hi: int, device):
    import torch

    i = torch.arange(n, dtype=torch.int64, device=device)
    width = max(1, hi // n)
    base = torch.div(i * hi, n, rounding_mode="floor")
    off = _srl_t(_hi32_t(n, seed, dist_id, 1, device) * width, 32)
    return torch.clamp(base + off, max=hi - 1)


def _as_u32_bits_t(v):
    """int64 values in [0, 2^32) -> int32 tensor with the same 32 bits."""
    import torch

    return torch.where(v >= 2**31, v - 2**32, v).to(torch.int32)


def keys_u32_torch(n: int, dist: int, seed: int = 0, device="cpu", chunk: int = 1 << 26):
    """keys_u32(n, dist, seed) built on `device` with torch (distributions
    0-6), the same bits as the numpy form, as an int32 tensor: for inputs
    too large to build on the host in good time."""
    import torch

    dist = int(dist)
    if dist in (0, 2):
        return u32_torch(n, seed, dist, device=device)
    if dist == 1:
        return _as_u32_bits_t(_uniform_below_t(n, 1000, seed, 1, 0, device))
    if dist in (3, 4, 5):
        a = _sorted_spread_t(n, seed, 3, 2**32, device)
        if dist == 4:
            a = torch.flip(a, dims=[0])
        elif dist == 5 and n // 100:
            # the swaps run one after another, as in the numpy form: replay
            # them on the host over the positions they touch
            m = n // 100
            xs = uniform_below(m, n, seed, 5, 2).astype(np.int64)
            ys = uniform_below(m, n, seed, 5, 3).astype(np.int64)
            pos = np.unique(np.concatenate([xs, ys]))
            vals = a[torch.from_numpy(pos).to(device)].cpu().numpy().tolist()
            where = {int(p): j for j, p in enumerate(pos.tolist())}
            for x, y in zip(xs.tolist(), ys.tolist()):
                jx, jy = where[x], where[y]
                vals[jx], vals[jy] = vals[jy], vals[jx]
            a[torch.from_numpy(pos).to(device)] = torch.tensor(vals, dtype=torch.int64, device=device)
        return _as_u32_bits_t(a)
    if dist == 6:
        out = torch.empty(n, dtype=torch.int32, device=device)
        for a0 in range(0, n, chunk):
            b0 = min(n, a0 + chunk)
            s = torch.zeros(b0 - a0, dtype=torch.int64, device=device)
            for j in range(6):
                d = u64_torch_range(a0, b0, seed, 6, 10 + j, device)
                s += _srl_t(d, 32)
                s += d & 0xFFFFFFFF
            v = 2**31 + ((s - 6 * 2**32) >> 12)
            out[a0:b0] = _as_u32_bits_t(torch.clamp(v, 0, 2**32 - 1))
        return out
    raise ValueError(f"no device form of distribution {dist}")


def keys_u64_shaped_torch(n: int, dist: int, seed: int = 0, device="cpu"):
    """keys_u64_shaped(n, dist, seed) built on `device` (int64 tensor, same
    bits)."""
    hi = keys_u32_torch(n, dist, seed, device).to(__import__("torch").int64) & 0xFFFFFFFF
    return (hi << 32) | _hi32_t(n, seed, 44, dist, device)


def keys_u64(n: int, key_bits: int = 64, seed: int = 0, dist_id: int = 20) -> np.ndarray:
    """n uint64 keys uniform over [0, 2^key_bits)."""
    d = u64(n, seed, dist_id)
    if key_bits < 64:
        d = d >> np.uint64(64 - key_bits)
    return d


def index_values(n: int) -> np.ndarray:
    """Payload = original index, so stability is visible in the output."""
    return np.arange(n, dtype=np.uint32)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int = 0, dist_id: int = 30) -> np.ndarray:
    """count sizes floor(exp(U(ln lo, ln hi))) (double precision; sizes only)."""
    d = u64(count, seed, dist_id)
    u = (d >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)
    s = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(s, lo, hi)


def unit_doubles(n: int, seed: int, dist_id: int, stream: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) from the top 53 bits of the draws."""
    return (u64(n, seed, dist_id, stream) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)


def poisson_arrivals(count: int, rate: float, seed: int = 0, dist_id: int = 40) -> np.ndarray:
    """Arrival times in seconds of a Poisson process of `rate` per second:
    cumulative sums of exponential gaps -ln(1 - u) / rate."""
    u = unit_doubles(count, seed, dist_id)
    return np.cumsum(-np.log1p(-u) / rate)


def served_mix(count: int, lo: int, hi: int, seed: int = 0):
    """Request mix of the served workload: (sizes log-uniform in [lo, hi],
    kind 0 = uint32 keys only (70%) or 1 = uint64 keys + uint32 values (30%),
    distribution id 0-6)."""
    sizes = log_uniform_sizes(count, lo, hi, seed=seed, dist_id=41)
    kind = (unit_doubles(count, seed, 42) >= 0.7).astype(np.int64)
    dist = uniform_below(count, 7, seed, 43).astype(np.int64)
    return sizes, kind, dist


def keys_u64_shaped(n: int, dist: int, seed: int = 0) -> np.ndarray:
    """uint64 keys with the shape of u32 distribution `dist` in their high
    half and uniform low halves: (keys_u32(n, dist) << 32) | draws."""
    hi = keys_u32(n, dist, seed).astype(np.uint64) << np.uint64(32)
    return hi | u32(n, seed, 44, dist).astype(np.uint64)


def segment_offsets(sizes) -> np.ndarray:
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.size + 1, np.uint64)
    off[1:] = np.cumsum(sizes).astype(np.uint64)
    return off
