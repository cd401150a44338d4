"""GPU parity of plans (one sort call captured into a CUDA graph and
replayed): every replay must equal the oracle, bit for bit, for radix,
bucket and segmented plans, with and without autotuning."""
import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kb,with_values,key_bits", [(4, False, 0), (4, True, 0), (8, False, 40), (8, True, 0)])
def test_radix_plan_replays_match_oracle(rs, oracle, kb, with_values, key_bits):
    import torch

    n = 300_001
    keys = synth.u32(n, 70, 0) if kb == 4 else synth.keys_u64(n, key_bits or 64, seed=71)
    vals = synth.index_values(n) if with_values else None
    kd = to_dev(keys)
    vd = to_dev(vals) if with_values else None
    ok = torch.empty_like(kd)
    ov = torch.empty_like(vd) if with_values else None
    plan = rs.Plan(rs.RS_PLAN_RADIX, kd, ok, vd, ov, key_bits=key_bits)
    kbits = key_bits or 8 * kb
    if with_values:
        wk, wv = oracle.radix_sort(keys, vals, kbits)
    else:
        wk, wv = oracle.radix_sort(keys, None, kbits), None
    cfg, nodes, ms = plan.info()
    assert nodes >= 2 and ms == -1.0 and cfg[0] > 0
    for rep in range(3):
        ok.zero_()
        plan.launch()
        torch.cuda.synchronize()
        assert_same(from_dev(ok, keys.dtype), wk, f"replay {rep} keys")
        if with_values:
            assert_same(from_dev(ov, np.uint32), wv, f"replay {rep} values")
    assert rs.get_status(plan.ws) == 0
    plan.close()


def test_radix_plan_follows_new_input_in_same_buffer(rs, oracle):
    """The graph reads the input buffer at replay time: new keys written into
    it are sorted by the next launch."""
    import torch

    n = 1 << 20
    kd = to_dev(synth.u32(n, 72, 0))
    ok = torch.empty_like(kd)
    plan = rs.Plan(rs.RS_PLAN_RADIX, kd, ok)
    for seed in (73, 74):
        keys = synth.keys_u32(n, 3, seed=seed)
        kd.copy_(to_dev(keys))
        plan.launch()
        torch.cuda.synchronize()
        assert_same(from_dev(ok, np.uint32), oracle.radix_sort(keys, None, 32), f"seed {seed}")
    plan.close()


def test_radix_plan_autotune_picks_a_compiled_shape(rs, oracle):
    import torch

    n = 2_000_003
    keys = synth.u32(n, 75, 0)
    kd = to_dev(keys)
    ok = torch.empty_like(kd)
    plan = rs.Plan(rs.RS_PLAN_RADIX, kd, ok, autotune=True)
    cfg, nodes, ms = plan.info()
    shapes = {rs.rs_config_get(4, False, i).as_tuple() for i in range(rs.rs_config_count(4, False))}
    assert cfg in shapes
    assert ms > 0.0
    ok.zero_()
    plan.launch()
    torch.cuda.synchronize()
    assert_same(from_dev(ok, np.uint32), oracle.radix_sort(keys, None, 32), "autotuned")
    # the second plan of the same class reuses the cached choice without timing
    plan2 = rs.Plan(rs.RS_PLAN_RADIX, kd, ok, autotune=True)
    cfg2, _, ms2 = plan2.info()
    assert cfg2 == cfg and ms2 == -1.0
    plan.close()
    plan2.close()


def test_radix_plan_in_place(rs, oracle):
    import torch

    n = 123_457
    keys = synth.keys_u64(n, 64, seed=76)
    kd = to_dev(keys)
    plan = rs.Plan(rs.RS_PLAN_RADIX, kd, kd)
    torch.cuda.synchronize()
    # creation ran the sort once already; write the input back and replay
    kd.copy_(to_dev(keys))
    plan.launch()
    torch.cuda.synchronize()
    assert_same(from_dev(kd, np.uint64), oracle.radix_sort(keys, None, 64), "in place")
    plan.close()


@pytest.mark.parametrize("dist,bounds", [(0, False), (4, True), (6, False)])
def test_bucket_plan_matches_oracle(rs, oracle, dist, bounds):
    import torch

    n = 500_000
    keys = synth.keys_u32(n, dist, seed=77)
    vals = synth.index_values(n)
    kd, vd = to_dev(keys), to_dev(vals)
    ok, ov = torch.empty_like(kd), torch.empty_like(vd)
    lo, hi = (int(keys.min()), int(keys.max())) if bounds else (1, 0)
    nb = 4096
    plan = rs.Plan(rs.RS_PLAN_BUCKET, kd, ok, vd, ov, min_key=lo, max_key=hi, num_buckets=nb)
    wk, wv = oracle.bucket_sort(keys, vals, int(keys.min()), int(keys.max()), nb)
    for rep in range(2):
        ok.zero_()
        ov.zero_()
        plan.launch()
        torch.cuda.synchronize()
        assert_same(from_dev(ok, np.uint32), wk, f"bucket replay {rep} keys")
        assert_same(from_dev(ov, np.uint32), wv, f"bucket replay {rep} values")
    assert rs.get_status(plan.ws) == 0
    plan.close()


@pytest.mark.parametrize("kb,with_values", [(4, False), (8, True)])
def test_segmented_plan_matches_oracle(rs, oracle, kb, with_values):
    import torch

    sizes = synth.log_uniform_sizes(400, 1, 120_000, seed=78)
    n = int(sizes.sum())
    keys = synth.u32(n, 79, 0) if kb == 4 else synth.keys_u64(n, 64, seed=79)
    vals = synth.index_values(n) if with_values else None
    off = synth.segment_offsets(sizes)
    kd = to_dev(keys)
    vd = to_dev(vals) if with_values else None
    od = to_dev(off.astype(np.uint64))
    ok = torch.empty_like(kd)
    ov = torch.empty_like(vd) if with_values else None
    plan = rs.Plan(rs.RS_PLAN_SEGMENTED, kd, ok, vd, ov, seg_offsets=od)
    _, nodes, _ = plan.info()
    assert nodes >= 3
    ok.zero_()
    plan.launch()
    torch.cuda.synchronize()
    if with_values:
        wk, wv = oracle.segmented_radix_sort(keys, off, vals, 8 * kb)
        assert_same(from_dev(ok, keys.dtype), wk, "segmented keys")
        assert_same(from_dev(ov, np.uint32), wv, "segmented values")
    else:
        assert_same(from_dev(ok, keys.dtype), oracle.segmented_radix_sort(keys, off, None, 8 * kb), "segmented")
    plan.close()


def test_plan_rejects_bad_arguments(rs):
    import torch

    kd = torch.zeros(1000, dtype=torch.int32, device="cuda")
    ok = torch.empty_like(kd)
    with pytest.raises(rs.SortError):
        rs.Plan(rs.RS_PLAN_RADIX, kd, ok, key_bits=33)
    desc = rs.RsPlanDesc(7, 4, kd.data_ptr(), ok.data_ptr(), None, None, 1000, 0, 1, 0, 0, None, 0, None, 0, 0)
    rc, h = rs.rs_plan_create(desc)
    assert rc == 1 and not h  # RS_ERR_INVALID_ARG


def test_segmented_plan_autotune_picks_a_compiled_shape(rs, oracle):
    import torch

    sizes = synth.log_uniform_sizes(200, 256, 300_000, seed=81)
    n = int(sizes.sum())
    keys = synth.u32(n, 82, 0)
    off = synth.segment_offsets(sizes)
    kd, od = to_dev(keys), to_dev(off.astype(np.uint64))
    ok = torch.empty_like(kd)
    plan = rs.Plan(rs.RS_PLAN_SEGMENTED, kd, ok, seg_offsets=od, autotune=True)
    cfg, nodes, ms = plan.info()
    shapes = {rs.rs_config_get(4, False, i).as_tuple()[1:] for i in range(rs.rs_config_count(4, False))}
    assert cfg[0] == 8 and cfg[1:] in shapes and ms > 0.0
    ok.zero_()
    plan.launch()
    torch.cuda.synchronize()
    assert_same(from_dev(ok, np.uint32), oracle.segmented_radix_sort(keys, off, None, 32), "autotuned segmented")
    plan.close()
