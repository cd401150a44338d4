"""GPU parity of typed-key sorts (rs_sort_typed): signed integers and
IEEE-754 floats, ascending and descending, keys only and with values, bit for
bit against the oracle's comparison sort."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

_UNSIGNED = {4: np.uint32, 8: np.uint64}


def _keys(dt, n, seed):
    """Random bit patterns of the dtype, plus its special values and repeats."""
    ut = _UNSIGNED[np.dtype(dt).itemsize]
    bits = synth.u64(n, seed, 50).astype(np.uint64)
    if ut is np.uint32:
        bits = bits >> np.uint64(32)
    x = bits.astype(ut).view(dt).copy()
    if np.issubdtype(dt, np.floating):
        # mostly ordinary numbers; random bit patterns are NaN-heavy for no gain
        x[: n // 2] = (synth.unit_doubles(n // 2, seed, 51) * 2 - 1).astype(dt) * dt(1e6)
        special = [np.nan, -np.nan, np.inf, -np.inf, 0.0, -0.0, 1.0, -1.0, np.finfo(dt).smallest_subnormal,
                   -np.finfo(dt).smallest_subnormal, np.finfo(dt).max, -np.finfo(dt).max]
    else:
        info = np.iinfo(dt)
        special = [info.min, info.max, -1, 0, 1, info.min + 1]
    m = min(n, len(special))
    x[:m] = np.array(special[:m], dt)
    if n > 40:
        x[n // 3: n // 3 + 20] = x[5]  # a run of one repeated key
    return x


def _to_dev(a):
    import torch

    signed = {4: np.int32, 8: np.int64}[a.dtype.itemsize]
    return torch.from_numpy(np.ascontiguousarray(a).view(signed)).cuda()


def _check(rs, oracle, dt, n, desc, with_values, in_place=False, seed=0):
    import torch

    x = _keys(dt, n, seed)
    ut = _UNSIGNED[x.dtype.itemsize]
    kind = 2 if np.issubdtype(dt, np.floating) else 1
    kd = _to_dev(x)
    vals = synth.index_values(n) if with_values else None
    vd = _to_dev(vals) if with_values else None
    if in_place:
        ok, ov = rs.sort_typed(kd, vd, kind=kind, descending=desc, out=kd, out_values=vd)
    else:
        ok, ov = rs.sort_typed(kd, vd, kind=kind, descending=desc)
    torch.cuda.synchronize()
    got = ok.cpu().numpy().view(ut)
    if with_values:
        wk, wv = oracle.sort_typed(x, vals, kind, desc)
        assert np.array_equal(ov.cpu().numpy().view(np.uint32), wv), "values differ"
    else:
        wk = oracle.sort_typed(x, None, kind, desc)
    want = wk.view(ut)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{dt.__name__} n={n} desc={desc}: {bad.size} differ, first at {bad[0]}")


@pytest.mark.parametrize("dt", [np.int32, np.int64, np.float32, np.float64])
@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("n", [3000, 250_001])
def test_typed_sort_matches_oracle(rs, oracle, dt, desc, n):
    _check(rs, oracle, dt, n, desc, with_values=False, seed=n)
    _check(rs, oracle, dt, n, desc, with_values=True, seed=n + 1)


@pytest.mark.parametrize("dt", [np.int32, np.float64])
def test_typed_sort_in_place(rs, oracle, dt):
    _check(rs, oracle, dt, 100_003, True, with_values=True, in_place=True, seed=9)
    _check(rs, oracle, dt, 2000, False, with_values=True, in_place=True, seed=10)


def test_unsigned_kind_descending(rs, oracle):
    import torch

    x = synth.u32(70_000, 11, 0)
    kd = _to_dev(x)
    ok, _ = rs.sort_typed(kd, kind=rs.RS_KEY_UINT, descending=True)
    torch.cuda.synchronize()
    assert np.array_equal(ok.cpu().numpy().view(np.uint32), oracle.sort_typed(x, None, 0, True))


def test_typed_rejects_bad_kind(rs):
    import torch

    kd = torch.zeros(10, dtype=torch.int32, device="cuda")
    ws = rs.workspace(rs.rs_workspace_bytes(0, 4, 0, 10, 0, 0, 0))
    assert rs.rs_sort_typed(7, 4, 0, kd, torch.empty_like(kd), None, None, 10, ws, ws.numel()) == 1
    assert rs.rs_sort_typed(1, 2, 0, kd, torch.empty_like(kd), None, None, 10, ws, ws.numel()) == 1
