#!/usr/bin/env python
"""Benchmark of the GPU integer sorts.

Default workload: LSD radix sort of 100,000,000 uint32 keys, uniform over
[0, 2^32), keys only, 8-bit digits (4 passes).  One step = one complete sort
call (digit counts + every scatter pass).  The keys (400 MB) are larger than
the 129 MB L2, so no L2 flush is needed between steps.

Prints ONE JSON line on rank 0: throughput (Gkeys/s, whole job), the
per-kernel roofline of the dominant kernel (its launches timed with CUDA
events on the launch stream during the timed region), the end-to-end rate
through the public API with host buffers, the clocks seen during the run, and
the CPU oracle timed on this host as a reported baseline.

--impl reference times the CPU oracle alone (the paper's sequential method)
on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank sorts its own array (replicas; the sort has
no exchange step), value = all keys / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gkeys/s & % HBM roofline at 100M u32; batched/served p50/p99 vs plain"
L2_BYTES = 129 * 2**20

WORKLOADS = {
    # name: (algo, key bytes, has values, n, key_bits, distribution, description)
    "radix_u32_100m": ("radix", 4, False, 100_000_000, 32, 0,
                       "LSD radix sort, 100M uint32 keys uniform [0,2^32), keys only, 8-bit digits, 4 passes"),
    "radix_u64kv_100m": ("radix", 8, True, 100_000_000, 64, None,
                         "LSD radix sort, 100M uint64 keys uniform [0,2^64) + uint32 index values, 8 passes"),
    "radix_u64_40bit_50m": ("radix", 8, False, 50_000_000, 40, None,
                            "LSD radix sort, 50M uint64 keys uniform [0,2^40), key_bits=40, 5 passes"),
}
# the seven 100M-key u32 distributions, radix (key_bits 32) and bucket (declared bounds, n/16 buckets)
for _d in range(7):
    _name = ["uniform", "small1000", "large", "sorted", "reverse", "nearly", "gauss"][_d]
    WORKLOADS[f"radix_u32_{_name}_100m"] = ("radix", 4, False, 100_000_000, 32, _d,
                                           f"LSD radix sort, 100M uint32 keys, distribution {_d}, 4 passes")
    WORKLOADS[f"bucket_u32_{_name}_100m"] = ("bucket", 4, False, 100_000_000, 32, _d,
                                            f"bucket sort, 100M uint32 keys, distribution {_d}, declared bounds, "
                                            f"n/16 buckets")
WORKLOADS["bucket_u32_1m"] = ("bucket", 4, False, 1_000_000, 31, 10,
                              "bucket sort, 1M uint32 keys uniform [0,2^31), 62,500 buckets over [0,2^31-1]")
WORKLOADS["radix_u32_1m"] = ("radix", 4, False, 1_000_000, 32, 10,
                             "LSD radix sort, 1M uint32 keys uniform [0,2^31), 8-bit digits, 4 passes")

# kernels whose algorithmic bytes per launch are 2 n (w + v) (one read and one
# write of every key) and n w (one read)
SCATTER_KERNELS = ("onesweep_pass", "bucket_pass", "onesweep_seg_pass", "local_sort")
READ_KERNELS = ("digit_counts", "seg_counts", "minmax")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="radix_u32_100m")
    ap.add_argument("--n", type=int, default=0, help="override the key count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("rs_onesweep.cuh", "rs_radix.cu", "rs_common.cuh"):
        with open(os.path.join(ROOT, "paper_1206_3511_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}@{workload}")
    if not e or e.get("source_sha") != kernel_source_sha():
        return None
    return e.get("dram_bytes_per_launch")


def make_keys(wl, n, seed=0):
    import numpy as np

    import synth

    algo, kb, has_v, _, key_bits, dist, _ = WORKLOADS[wl]
    if kb == 4:
        if dist == 10:  # uniform [0, 2^31)
            keys = synth.keys_u32(n, 0, seed=seed) >> np.uint32(1)
        else:
            keys = synth.keys_u32(n, dist, seed=seed)
    else:
        keys = synth.keys_u64(n, key_bits, seed=seed)
    vals = synth.index_values(n) if has_v else None
    return keys, vals


def bucket_bounds(wl):
    import synth

    dist = WORKLOADS[wl][5]
    if dist == 10:
        return 0, 2**31 - 1
    return synth.DECLARED_BOUNDS[dist]


def cpu_oracle_rate(wl, n_sample, keys=None, vals=None) -> tuple[float, float]:
    """The oracle's sort of n_sample keys of the workload (radix, or bucket
    for bucket workloads): (Gkeys/s, seconds)."""
    import oracle

    if keys is None:
        keys, vals = make_keys(wl, n_sample, seed=1)
    algo, _, _, _, key_bits, _, _ = WORKLOADS[wl]
    t0 = time.perf_counter()
    if algo == "bucket":
        lo, hi = bucket_bounds(wl)
        oracle.bucket_sort(keys, vals, lo, hi, max(1, keys.size // 16))
    else:
        oracle.radix_sort(keys, vals, key_bits, 8)
    dt = time.perf_counter() - t0
    return keys.size / dt / 1e9, dt


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    wl = args.workload
    n_full = args.n or WORKLOADS[wl][3]
    # each step sorts a bounded sample so that the whole run stays within a
    # few minutes: about 90 s of oracle work spread over warmup + steps
    total_steps = max(1, args.warmup + args.steps)
    n_sample = int(min(n_full, max(500_000, min(10_000_000, 90 * 20_000_000 // total_steps))))
    import oracle

    oracle.build()
    keys, vals = make_keys(wl, n_sample, seed=1)
    rates = []
    for i in range(total_steps):
        r, _ = cpu_oracle_rate(wl, n_sample, keys, vals)
        if i >= args.warmup:
            rates.append(r)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": n_sample / value / 1e6,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": _dtype(wl),
        "data": "synthetic",
        "config": {"workload": WORKLOADS[wl][6], "n": n_full, "parallelism": "none (1 CPU thread)"},
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_sample} keys of the workload per step, single-threaded C oracle "
                                   f"(LSD radix, 8-bit digits), {os.cpu_count()} host cores present"},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _dtype(wl):
    return "u32" if WORKLOADS[wl][1] == 4 else "u64"


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_1206_3511_gb300 as rs

    world, rank, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    rs.load()
    wl = args.workload
    algo, kb, has_v, n_def, key_bits, _, desc = WORKLOADS[wl]
    if algo == "bucket":
        key_bits = 8 * kb
    n = args.n or n_def
    keys_np, vals_np = make_keys(wl, n, seed=rank)
    sdt = np.int32 if kb == 4 else np.int64
    h_keys = torch.from_numpy(keys_np.view(sdt)).pin_memory()
    h_vals = torch.from_numpy(vals_np.view(np.int32)).pin_memory() if has_v else None
    d_keys = h_keys.to(dev, non_blocking=False)
    d_vals = h_vals.to(dev) if has_v else None
    d_out = torch.empty_like(d_keys)
    d_outv = torch.empty_like(d_vals) if has_v else None
    stream = torch.cuda.current_stream()
    if algo == "bucket":
        lo, hi = bucket_bounds(wl)
        nb = max(1, n // 16)
        nbytes = rs.rs_workspace_bytes(rs.RS_ALGO_BUCKET, kb, has_v, n, 0, nb, 0)
        bfn = rs.bs_sort_u32 if kb == 4 else rs.bs_sort_u64

        def call(ws):
            return bfn(d_keys, d_out, d_vals, d_outv, n, lo, hi, nb, ws, ws.numel(), stream)
    else:
        nbytes = rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, kb, has_v, n, key_bits, 0, 0)
        rfn = rs.rs_sort_u32 if kb == 4 else rs.rs_sort_u64

        def call(ws):
            return rfn(d_keys, d_out, d_vals, d_outv, n, key_bits, ws, ws.numel(), stream)
    ws = rs.workspace(nbytes, d_keys.device)

    def step():
        rc = call(ws)
        if rc:
            raise rs.SortError(rc, "sort")

    sampler = ClockSampler(dev)
    sampler.start()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    rs.rs_profile_enable(True)
    launches0 = rs.rs_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches = rs.rs_launch_count() - launches0
    rs.rs_profile_enable(False)
    kstats = rs.rs_profile_read()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    status = rs.get_status(ws)
    if status:
        raise rs.SortError(status, "device status after the timed steps")

    # correctness spot check of the last result (full check lives in the tests)
    chk = d_out[: min(n, 1 << 20)]
    if kb == 4:
        a = chk.cpu().numpy().view(np.uint32)
    else:
        a = chk.cpu().numpy().view(np.uint64)
    assert np.all(a[1:] >= a[:-1]), "bench output not sorted"

    # end to end through the public API: pinned host keys -> device -> sort -> host
    h_out = torch.empty_like(h_keys).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        d_keys.copy_(h_keys, non_blocking=True)
        step()
        h_out.copy_(d_out, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        d_keys.copy_(h_keys, non_blocking=True)
        if has_v:
            d_vals.copy_(h_vals, non_blocking=True)
        step()
        h_out.copy_(d_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    if world > 1:
        t = torch.tensor([ms, e2e_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, e2e_ms = float(t[0]), float(t[1])
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    value = world * n * args.steps / (ms / 1e3) / 1e9
    e2e_value = world * n * e2e_steps / (e2e_ms / 1e3) / 1e9
    h2d = n * kb + (n * 4 if has_v else 0)
    d2h = n * kb

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    w = kb + (4 if has_v else 0)
    # dominant kernel by time inside the timed region: its algorithmic bytes
    # per step over its device time per step (for a kernel launched once per
    # pass this is bytes per launch over the mean launch time)
    roofline = None
    if kstats:
        top = max(kstats, key=lambda k: kstats[k][1])
        nl, tot = kstats[top]
        per_step_launches = nl / args.steps
        if top == "onesweep_pass":
            step_bytes = 2 * n * w * per_step_launches
        elif top in SCATTER_KERNELS:
            step_bytes = 2 * n * w  # the launches of one step move every key once
        else:
            step_bytes = n * kb * per_step_launches
        step_s = tot / args.steps / 1e3
        achieved = step_bytes / step_s / 1e9
        traffic = ncu_traffic(top, wl)
        roofline = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": f"{peak_src} copy bandwidth",
                    "algorithmic_bytes_per_launch": step_bytes / per_step_launches,
                    "avg_launch_ms": tot / nl, "launches": nl}
    if algo == "bucket":
        # one read to count, one read+write to scatter into buckets, one
        # read+write to sort the buckets
        whole_bytes = n * kb + 4 * n * w
    else:
        passes = -(-key_bits // 8)
        whole_bytes = n * kb + passes * 2 * n * w
    step_s = ms / args.steps / 1e3
    whole = {"algorithmic_bytes_per_step": whole_bytes,
             "achieved_gbs": whole_bytes / step_s / 1e9,
             "frac_of_peak": whole_bytes / step_s / 1e9 / hbm_peak,
             "kernels": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kstats.items()}}

    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        n_sample = n
        rate, secs = cpu_oracle_rate(wl, n_sample)
        cpu = {"value": rate, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle sort of {n_sample} keys of the same workload ({secs:.1f} s), "
                         f"single thread of {os.cpu_count()} host cores"}

    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(wl), "data": "synthetic",
        "config": {"workload": desc, "n": n, "key_bits": key_bits, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (%d MB keys vs 129 MB L2), no flush" % (n * kb // 2**20)},
        "clocks": clocks, "gpu_launches": launches, "roofline": roofline, "whole_sort": whole,
        "e2e": {"value": e2e_value, "unit": "Gkeys/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
