"""The workspace-free entry point rs_sort_u32_noalloc, for callers that cannot
allocate device memory: its results must equal rs_sort_u32's and the CPU
oracle's (exactly: this is integer work) on two calls in a row that reuse the
library's shared scratch, sizes above its cap must be refused before anything
is enqueued, and its argument rules must be rs_sort_u32's (also at n = 0).

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.  It also passes on its own in a
fresh process."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _with_workspace(rs, keys, vals, key_bits):
    import torch

    kd = to_dev(keys)
    vd = to_dev(vals) if vals is not None else None
    out = torch.empty_like(kd)
    outv = torch.empty_like(vd) if vd is not None else None
    ws = rs.workspace(rs.rs_workspace_bytes(0, 4, vals is not None, keys.size, key_bits, 0, 0))
    assert rs.rs_sort_u32(kd, out, vd, outv, keys.size, key_bits, ws, ws.numel()) == 0
    torch.cuda.synchronize()
    return from_dev(out, np.uint32), (from_dev(outv, np.uint32) if vals is not None else None)


def _no_alloc(rs, keys, vals, key_bits):
    import torch

    kd = to_dev(keys)
    vd = to_dev(vals) if vals is not None else None
    out = torch.full_like(kd, -1)
    outv = torch.full_like(vd, -1) if vd is not None else None
    assert rs.rs_sort_u32_noalloc(kd, out, vd, outv, keys.size, key_bits) == 0
    torch.cuda.synchronize()
    return from_dev(out, np.uint32), (from_dev(outv, np.uint32) if vals is not None else None)


@pytest.mark.parametrize("with_values", [False, True])
def test_no_alloc_matches_workspace_sort_twice(rs, oracle, with_values):
    from paper_1206_3511_gb300 import _lib

    cap = _lib.RS_NOALLOC_MAX_KEYS
    for call, (n, dist, key_bits) in enumerate([(300_007, 0, 32), (cap, 6, 32)]):
        keys = synth.keys_u32(n, dist, seed=11 + call)
        vals = synth.index_values(n) if with_values else None
        want_k, want_v = _with_workspace(rs, keys, vals, key_bits)
        got_k, got_v = _no_alloc(rs, keys, vals, key_bits)
        assert_same(got_k, want_k, f"no-alloc keys vs rs_sort_u32, call {call}")
        if with_values:
            assert_same(got_v, want_v, f"no-alloc values vs rs_sort_u32, call {call}")
            ok, ov = oracle.radix_sort(keys, vals, key_bits)
            assert_same(got_k, ok, f"no-alloc keys vs oracle, call {call}")
            assert_same(got_v, ov, f"no-alloc values vs oracle, call {call}")
        else:
            assert_same(got_k, oracle.radix_sort(keys, None, key_bits), f"no-alloc keys vs oracle, call {call}")


def test_no_alloc_refuses_sizes_above_its_cap(rs):
    import torch

    from paper_1206_3511_gb300 import _lib

    n = _lib.RS_NOALLOC_MAX_KEYS + 1
    kd = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty_like(kd)
    assert rs.rs_sort_u32_noalloc(kd, out, None, None, n, 32) == 1  # RS_ERR_INVALID_ARG
    assert rs.rs_sort_u32_noalloc(None, None, None, None, 0, 32) == 0  # n = 0 is a no-op


def test_no_alloc_argument_rules_equal_rs_sort_u32_at_n_zero(rs):
    """At n = 0 both calls check key_bits and the pairing of the value
    pointers before returning."""
    import torch

    v = torch.zeros(4, dtype=torch.int32, device="cuda")
    ws = rs.workspace(4096)
    for key_bits, vi, vo in [(40, None, None), (32, v, None), (32, None, v), (0, None, None), (32, v, v)]:
        want = rs.rs_sort_u32(None, None, vi, vo, 0, key_bits, ws, ws.numel())
        assert rs.rs_sort_u32_noalloc(None, None, vi, vo, 0, key_bits) == want, (key_bits, vi is None, vo is None)
    assert rs.rs_sort_u32_noalloc(None, None, None, None, 0, 40) == 1
