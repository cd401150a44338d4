"""The multi-process path of the benchmark on CPU (gloo, two ranks): the
job's time is the slowest rank's, the job's rate counts every rank's keys,
and every rank sorts its own seeded inputs (replicas, weak scaling)."""
import os
import socket

import numpy as np
import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        env = bench._dist_env()
        # rank r took (r + 1) ms for the sort and (10 - r) ms end to end
        times = bench.max_over_ranks([rank + 1.0, 10.0 - rank])
        keys, _ = bench.make_keys("radix_u32_1m", 1000, seed=env[1])
        q.put((rank, env, times, keys.tolist()))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, "error", repr(e), None))


def test_two_gloo_ranks_take_the_slowest_time_and_sort_their_own_inputs():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, env, times, keys = q.get(timeout=120)
        assert env != "error", times
        out[rank] = (env, times, keys)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == (2, 0, 0) and out[1][0] == (2, 1, 1)
    assert out[0][1] == [2.0, 10.0] and out[1][1] == [2.0, 10.0]  # max over ranks on every rank
    assert out[0][2] != out[1][2]  # each rank's own seeded keys


def test_job_rate_counts_every_rank():
    import bench

    # 2 ranks x 100M keys in 2 ms (the slowest rank) = 100 Gkeys/s for the job
    assert bench.job_rate(100_000_000, 2, 2.0) == pytest.approx(100.0)
    assert bench.job_rate(100_000_000, 1, 2.0) == pytest.approx(50.0)


def test_single_process_max_is_identity():
    import bench

    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert np.isfinite(bench.job_rate(1, 1, 1.0))


def test_link_bound_is_the_slowest_stage():
    import bench

    rates = {"h2d_gbs": 200.0, "d2h_gbs": 190.0, "both_gbs": 333.0}
    # 100M u32 keys: 400 MB each way; both directions share 333 GB/s -> 2.4 ms
    assert bench.link_bound(100_000_000, 4e8, 4e8, 2.1, rates) == pytest.approx(100e6 / (8e8 / 333e9) / 1e9)
    # a sort slower than the copies sets the bound
    assert bench.link_bound(100_000_000, 4e8, 4e8, 5.0, rates) == pytest.approx(20.0)
    # one direction alone can be the bound
    assert bench.link_bound(1, 1.9e9, 0, 0.0, rates) == pytest.approx(1 / (1.9e9 / 200e9) / 1e9)


def test_traffic_is_used_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    import json

    import bench

    sha = bench.kernel_source_sha("onesweep_pass")
    assert len(sha) == 16 and sha != bench.kernel_source_sha("onesweep_seg_pass")
    p = tmp_path / "profiles"
    p.mkdir()
    (p / "traffic.json").write_text(json.dumps({
        "onesweep_pass@w": {"dram_bytes_per_launch": 123, "source_sha": sha},
        "onesweep_seg_pass@w": {"dram_bytes_per_launch": 456, "source_sha": "stale"}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_1206_3511_gb300" / "csrc"
    csrc.mkdir(parents=True)
    import os
    import shutil

    real = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1206_3511_gb300", "csrc")
    for f in set(bench.KERNEL_SOURCES["onesweep_pass"]) | set(bench.KERNEL_SOURCES["onesweep_seg_pass"]):
        shutil.copy(os.path.join(real, f), csrc / f)
    assert bench.ncu_traffic("onesweep_pass", "w") == 123
    assert bench.ncu_traffic("onesweep_seg_pass", "w") is None   # taken on other sources
    assert bench.ncu_traffic("digit_counts", "w") is None        # no entry
    with open(csrc / "rs_radix.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.ncu_traffic("onesweep_pass", "w") is None       # its kernel changed since
