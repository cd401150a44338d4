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
                            "LSD radix sort, 50M uint64 keys uniform [0,2^40), key_bits=40, autotuned digit width "
                            "and kernel shape"),
}
# the seven 100M-key u32 distributions, radix (key_bits 32) and bucket (declared bounds, n/16 buckets)
for _d in range(7):
    _name = ["uniform", "small1000", "large", "sorted", "reverse", "nearly", "gauss"][_d]
    WORKLOADS[f"radix_u32_{_name}_100m"] = ("radix", 4, False, 100_000_000, 32, _d,
                                           f"LSD radix sort, 100M uint32 keys, distribution {_d}, 4 passes")
    WORKLOADS[f"bucket_u32_{_name}_100m"] = ("bucket", 4, False, 100_000_000, 32, _d,
                                            f"bucket sort, 100M uint32 keys, distribution {_d}, declared bounds, "
                                            f"n/16 buckets")
WORKLOADS["bucket_u64_uniform_100m"] = ("bucket", 8, False, 100_000_000, 64, 20,
                                        "bucket sort, 100M uint64 keys uniform [0,2^64), bounds computed on the "
                                        "device (min and max of the keys), n/16 buckets")
WORKLOADS["bucket_u32_1m"] = ("bucket", 4, False, 1_000_000, 31, 10,
                              "bucket sort, 1M uint32 keys uniform [0,2^31), 62,500 buckets over [0,2^31-1]")
WORKLOADS["radix_u32_1m"] = ("radix", 4, False, 1_000_000, 32, 10,
                             "LSD radix sort, 1M uint32 keys uniform [0,2^31), 8-bit digits, 4 passes")
WORKLOADS["paper_cases"] = ("paper", 4, False, 100_000_000, 0, None,
                            "the paper's six input cases (Sec. 3.1) at n = 10^6, 10^7, 10^8: radix sort with key_bits "
                            "= bit length of M - 1 and bucket sort with bounds [0, M - 1] and n/16 buckets")
# the paper's Table 1: seconds on a laptop (Intel i5), sequential C++, per case: radix at n = 10^6, 10^7, 10^8, then
# bucket at the same sizes (context only)
PAPER_TABLE1_S = {
    1: (1.78, 17.66, 176.84, 0.74, 5.84, 45.92),
    2: (1.88, 18.93, 174.85, 0.61, 4.14, 26.83),
    3: (1.86, 17.69, 178.68, 0.61, 4.12, 28.27),
    4: (1.05, 11.10, 105.31, 0.31, 3.00, 31.54),
    5: (2.45, 24.56, 246.28, 0.78, 8.54, 97.43),
    6: (1.77, 17.66, 176.65, 0.61, 5.18, 41.06),
}
# n = number of arrays (batched) or requests per arrival rate (served)
WORKLOADS["batched_u32_20k"] = ("batched", 4, False, 20_000, 32, 0,
                                "segmented sort of 20,000 uint32 arrays, sizes log-uniform in [256, 2,000,000] "
                                "(seed 0), uniform keys, one CUDA-graph launch with the autotuned pass shape; "
                                "vs one rs_sort_u32 call per array")
WORKLOADS["batched_u32_tiny"] = ("batched", 4, False, 200_000, 32, 0,
                                 "segmented sort of 200,000 uint32 arrays, sizes log-uniform in [1, 256] (seed 0), "
                                 "uniform keys, one CUDA-graph launch; vs one rs_sort_u32 call per array")
WORKLOADS["served_mix"] = ("served", 4, False, 1_000, 32, None,
                           "sort server: Poisson arrivals at 1k-50k req/s, sizes log-uniform in [1e3, 5e7] keys, "
                           "70% uint32 keys-only / 30% uint64 keys + uint32 values, distributions 0-6, 80 GB budget; "
                           "vs a FIFO of one sort per request on one stream")
BATCH_LO, BATCH_HI = 256, 2_000_000
# size law of each batched workload: log-uniform in [lo, hi]
BATCH_SIZES = {"batched_u32_20k": (BATCH_LO, BATCH_HI), "batched_u32_tiny": (1, 256)}
SERVED_LO, SERVED_HI = 1_000, 50_000_000
SERVED_RATES = (1_000, 2_000, 5_000, 10_000, 20_000, 35_000, 50_000)
SERVED_BUDGET = 80 * 10**9

# radix workloads whose kernel shape and digit width come from the autotuner
AUTOTUNED = ("radix_u64_40bit_50m",)

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
    ap.add_argument("--autotune", action="store_true", help="radix: pick the kernel shape with the autotuner")
    ap.add_argument("--no-context", action="store_true", help="skip the torch.sort context timing")
    ap.add_argument("--no-batched-served", dest="batched_served", action="store_false",
                    help="default workload: skip the batched and served comparisons added to the line")
    ap.add_argument("--rates", default="", help="served: comma-separated arrival rates per second")
    ap.add_argument("--no-bucket-sweep", dest="bucket_sweep", action="store_false",
                    help="served: skip the second sweep with half the requests bucket sorts")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Context only: a library radix sort (CUB's DeviceRadixSort::SortKeys, from
# the CUDA toolkit's headers) of the same keys on the same GPU, compiled on
# the fly into a temporary directory.
_CUB_SRC = r"""
#include <cub/device/device_radix_sort.cuh>
#include <cstdint>
extern "C" int cub_sort_keys_u32(const uint32_t* in, uint32_t* out, size_t n, void* tmp, size_t* tmp_bytes,
                                 cudaStream_t s) {
    return (int)cub::DeviceRadixSort::SortKeys(tmp, *tmp_bytes, in, out, (int)n, 0, 32, s);
}
"""


def cub_context(d_keys, n, stream, reps=20):
    """Gkeys/s of CUB's keys-only radix sort of d_keys (u32), or None."""
    import ctypes
    import shutil
    import tempfile

    import torch

    try:
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = tempfile.mkdtemp(prefix="cubctx")
        src, lib = os.path.join(tmp, "cub_sort.cu"), os.path.join(tmp, "libcubsort.so")
        with open(src, "w") as f:
            f.write(_CUB_SRC)
        inc = [f"-I{d}" for d in ("/usr/local/cuda/include/cccl",) if os.path.isdir(d)]
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O3", "-Xcompiler",
                        "-fPIC", "-shared", *inc, "-o", lib, src], check=True, capture_output=True, timeout=300)
        cub = ctypes.CDLL(lib)
        cub.cub_sort_keys_u32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p]
        out = torch.empty_like(d_keys)
        nbytes = ctypes.c_size_t(0)
        if cub.cub_sort_keys_u32(d_keys.data_ptr(), out.data_ptr(), n, None, ctypes.byref(nbytes), None):
            return None
        tmpbuf = torch.empty(nbytes.value, dtype=torch.uint8, device=d_keys.device)

        def run():
            return cub.cub_sort_keys_u32(d_keys.data_ptr(), out.data_ptr(), n, tmpbuf.data_ptr(), ctypes.byref(nbytes),
                                         stream.cuda_stream)

        for _ in range(3):
            if run():
                return None
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            run()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        return {"value": n / (ms / 1e3) / 1e9, "unit": "Gkeys/s", "ms_per_sort": ms,
                "note": "cub::DeviceRadixSort::SortKeys (CUDA toolkit), uint32 keys only, same keys and GPU"}
    except Exception:
        return None


# End-to-end loops per mode; the median is reported.  The host link is shared
# with other work on the machine, and single loops have run at half speed.
E2E_REPEATS = 5


def pass_bytes(n, key_bytes, has_values) -> int:
    """Algorithmic HBM bytes of one scatter pass: every key (and value) read
    once and written once."""
    return 2 * n * (key_bytes + (4 if has_values else 0))


def sort_bytes(algo, n, key_bytes, has_values, key_bits=0, digit_bits=8, bounds_computed=False) -> int:
    """Algorithmic HBM bytes of one whole sort.  Radix: one read of the keys
    to count every digit, then one read and one write of keys (and values)
    per pass.  Bucket: one read to count, then a read and a write to scatter
    into buckets and another to sort the buckets, plus one read of the keys
    for their min and max when the bounds are not declared."""
    if algo == "bucket":
        return (2 if bounds_computed else 1) * n * key_bytes + 2 * pass_bytes(n, key_bytes, has_values)
    passes = -(-(key_bits or 8 * key_bytes) // digit_bits)
    return n * key_bytes + passes * pass_bytes(n, key_bytes, has_values)


def host_link_rates(h_src, h_dst, d_a, d_b, reps=3) -> dict:
    """Copy rates of the host link on the step's own pinned buffers: host to
    device alone, device to host alone, and both at once on two streams
    (GB/s, median of reps).  The copied size is that of h_src, up to 1 GB."""
    import torch

    nb = min(h_src.numel() * h_src.element_size(), 1 << 30)
    hs, hd = h_src.view(torch.uint8)[:nb], h_dst.view(torch.uint8)[:nb]
    da, db = d_a.view(torch.uint8)[:nb], d_b.view(torch.uint8)[:nb]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cur = torch.cuda.current_stream()
            e0.record(cur)
            s1.wait_event(e0)
            s2.wait_event(e0)
            fn()
            for s in (s1, s2):
                d = torch.cuda.Event()
                d.record(s)
                cur.wait_event(d)
            e1.record(cur)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts[1:])[len(ts[1:]) // 2] / 1e3

    def h2d():
        with torch.cuda.stream(s1):
            da.copy_(hs, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            hd.copy_(db, non_blocking=True)

    def both():
        h2d()
        d2h()

    return {"h2d_gbs": nb / timed(h2d) / 1e9, "d2h_gbs": nb / timed(d2h) / 1e9,
            "both_gbs": 2 * nb / timed(both) / 1e9}


def link_bound(units, h2d_bytes, d2h_bytes, sort_ms, rates) -> float:
    """Throughput ceiling of the pipelined end-to-end steps: a step takes at
    least the longest of its sort, its upload, its download and both copies
    sharing the link (units per second / 1e9)."""
    t = max(sort_ms / 1e3, h2d_bytes / (rates["h2d_gbs"] * 1e9), d2h_bytes / (rates["d2h_gbs"] * 1e9),
            (h2d_bytes + d2h_bytes) / (rates["both_gbs"] * 1e9))
    return units / t / 1e9


def max_over_ranks(values, device=None) -> list[float]:
    """Each value's maximum over all ranks (the job's time is its slowest
    rank's); the values themselves on a single process."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(units_per_rank: float, world: int, ms: float, scale: float = 1e9) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time
    (weak scaling: each rank sorts its own inputs)."""
    return world * units_per_rank / (ms / 1e3) / scale


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


# the sources that define each kernel whose DRAM traffic profiles/traffic.json
# records; a recorded figure is used only while these files are unchanged
KERNEL_SOURCES = {
    "onesweep_pass": ("rs_onesweep.cuh", "rs_common.cuh", "rs_radix.cu", "rs_radix.h"),
    "onesweep_seg_pass": ("rs_onesweep.cuh", "rs_common.cuh", "rs_segmented.cuh", "rs_segmented.cu",
                          "rs_segmented.h"),
}


def kernel_source_sha(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1206_3511_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}@{workload}")
    if not e or e.get("source_sha") != kernel_source_sha(kernel):
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
    """Declared (min, max) of a bucket workload; (1, 0) = computed on the device."""
    import synth

    kb, dist = WORKLOADS[wl][1], WORKLOADS[wl][5]
    if kb == 8:
        return 1, 0
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
        if lo > hi:  # bounds computed from the keys
            lo = hi = None
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
    tuned = None
    if algo == "bucket":
        lo, hi = bucket_bounds(wl)
        nb = max(1, n // 16)
        nbytes = rs.rs_workspace_bytes(rs.RS_ALGO_BUCKET, kb, has_v, n, 0, nb, 0)
        bfn = rs.bs_sort_u32 if kb == 4 else rs.bs_sort_u64

        def sort_into(kin, kout, vin, vout, ws, strm):
            return bfn(kin, kout, vin, vout, n, lo, hi, nb, ws, ws.numel(), strm)

        def call(ws):
            return sort_into(d_keys, d_out, d_vals, d_outv, ws, stream)
    else:
        if args.autotune or wl in AUTOTUNED:
            # the plan's autotuner picks the kernel shape and digit width; the
            # timed calls then use that shape (eager, so kernels are timed)
            plan = rs.Plan(rs.RS_PLAN_RADIX, d_keys, d_out, d_vals, d_outv, key_bits=key_bits, autotune=True)
            tuned, _, tuned_ms = plan.info()
            plan.close()
            nbytes = rs.rs_workspace_bytes_cfg(kb, has_v, n, key_bits, tuned)
        else:
            nbytes = rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, kb, has_v, n, key_bits, 0, 0)
        rfn = rs.rs_sort_u32_ex if kb == 4 else rs.rs_sort_u64_ex

        def sort_into(kin, kout, vin, vout, ws, strm):
            return rfn(kin, kout, vin, vout, n, key_bits, ws, ws.numel(), strm, tuned)

        def call(ws):
            return sort_into(d_keys, d_out, d_vals, d_outv, ws, stream)
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
    ms = ev0.elapsed_time(ev1)
    # per-kernel times: the same steps again with CUDA events recorded on the
    # launch stream around every launch (kept out of the timed region above,
    # where their host cost would add to short sorts)
    prof_steps = args.steps
    rs.rs_profile_enable(True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    rs.rs_profile_enable(False)
    kstats = rs.rs_profile_read()
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

    # end to end through the host-buffer C calls (rs_sort_host_* /
    # bs_sort_host_*): every step copies its keys (and values) from pinned
    # host memory into a device buffer, sorts them there and copies the sorted
    # keys (and values) back, all inside one library call.  Serial: one
    # stream, nothing overlaps.
    e2e_steps = max(3, min(args.steps, 20))
    if algo == "bucket":
        hbytes = rs.rs_host_sort_bytes(rs.RS_ALGO_BUCKET, kb, has_v, n, 0, nb)
        hfn = rs.bs_sort_host_u32 if kb == 4 else rs.bs_sort_host_u64

        def host_call(hk_out, hv_out, buf, strm):
            return hfn(h_keys, hk_out, h_vals, hv_out, n, lo, hi, nb, buf, buf.numel(), strm)
    else:
        hbytes = rs.rs_host_sort_bytes(rs.RS_ALGO_RADIX, kb, has_v, n, key_bits, 0)
        hfn = rs.rs_sort_host_u32 if kb == 4 else rs.rs_sort_host_u64

        def host_call(hk_out, hv_out, buf, strm):
            return hfn(h_keys, hk_out, h_vals, hv_out, n, key_bits, buf, buf.numel(), strm)

    S = 3
    hbufs = [rs.workspace(hbytes, d_keys.device) for _ in range(S)]
    houts = [torch.empty_like(h_keys).pin_memory() for _ in range(S)]
    houtv = [torch.empty_like(h_vals).pin_memory() if has_v else None for _ in range(S)]

    def host_step(j, strm):
        rc = host_call(houts[j], houtv[j], hbufs[j], strm)
        if rc:
            raise rs.SortError(rc, "host-buffer sort")

    for _ in range(2):
        host_step(0, stream)
    torch.cuda.synchronize()

    def serial_run():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            host_step(0, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    serial_all = [serial_run() for _ in range(E2E_REPEATS)]
    e2e_serial_ms = float(np.median(serial_all))
    h_out = houts[0].clone()

    # Pipelined: successive calls go round-robin to three streams, each with
    # its own device buffer and host output, so that one call's upload and
    # another's download run while a third sorts (how a stream of sort jobs
    # is served).  Calls on one stream run in order.
    hstreams = [torch.cuda.Stream() for _ in range(S)]
    for j in range(S):
        host_step(j, hstreams[j])
    torch.cuda.synchronize()

    def pipe_run():
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for hs in hstreams:
            hs.wait_event(p0)
        for i in range(e2e_steps):
            host_step(i % S, hstreams[i % S])
        for hs in hstreams:
            done = torch.cuda.Event()
            done.record(hs)
            stream.wait_event(done)
        p1.record(stream)
        torch.cuda.synchronize()
        return p0.elapsed_time(p1)

    pipe_all = [pipe_run() for _ in range(E2E_REPEATS)]
    e2e_ms = float(np.median(pipe_all))
    for j in range(S):
        assert rs.get_status(hbufs[j]) == 0
        assert torch.equal(houts[j], h_out), "pipelined result differs from the serial one"
    link = host_link_rates(h_keys, houts[1], d_out, d_keys)  # overwrites houts[1] and d_out

    ms, e2e_ms, e2e_serial_ms = max_over_ranks([ms, e2e_ms, e2e_serial_ms], device=dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    value = job_rate(n * args.steps, world, ms)
    e2e_value = job_rate(n * e2e_steps, world, e2e_ms)
    e2e_serial = job_rate(n * e2e_steps, world, e2e_serial_ms)
    h2d = n * kb + (n * 4 if has_v else 0)
    d2h = n * kb + (n * 4 if has_v else 0)

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    # dominant kernel by time inside the timed region: its algorithmic bytes
    # per step over its device time per step (for a kernel launched once per
    # pass this is bytes per launch over the mean launch time)
    roofline = None
    if kstats:
        top = max(kstats, key=lambda k: kstats[k][1])
        nl, tot = kstats[top]
        per_step_launches = nl / prof_steps
        if top == "onesweep_pass":
            step_bytes = pass_bytes(n, kb, has_v) * per_step_launches
        elif top in SCATTER_KERNELS:
            step_bytes = pass_bytes(n, kb, has_v)  # the launches of one step move every key once
        else:
            step_bytes = n * kb * per_step_launches
        step_s = tot / prof_steps / 1e3
        achieved = step_bytes / step_s / 1e9
        traffic = ncu_traffic(top, wl)
        roofline = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": f"{peak_src} copy bandwidth",
                    "algorithmic_bytes_per_launch": step_bytes / per_step_launches,
                    "avg_launch_ms": tot / nl, "launches": nl,
                    "timing": f"CUDA events around every launch over a repeat of the {prof_steps} timed steps"}
    whole_bytes = sort_bytes(algo, n, kb, has_v, key_bits, tuned[0] if (tuned and algo == "radix") else 8,
                             bounds_computed=algo == "bucket" and lo > hi)
    step_s = ms / args.steps / 1e3
    whole = {"algorithmic_bytes_per_step": whole_bytes,
             "achieved_gbs": whole_bytes / step_s / 1e9,
             "frac_of_peak": whole_bytes / step_s / 1e9 / hbm_peak,
             "kernels": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kstats.items()}}

    # context: a library sort (torch.sort, stable, keys only) of the same
    # keys on the same GPU, read as signed integers of the same width
    lib = None
    if not args.no_context:
        t_in = d_keys.clone()
        for _ in range(2):
            torch.sort(t_in, stable=True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        c0.record(stream)
        for _ in range(reps):
            torch.sort(t_in, stable=True)
        c1.record(stream)
        torch.cuda.synchronize()
        lib_ms = c0.elapsed_time(c1) / reps
        lib = {"torch.sort": {"value": n / (lib_ms / 1e3) / 1e9, "unit": "Gkeys/s", "ms_per_sort": lib_ms,
                              "note": "stable torch.sort of the keys as signed integers (returns indices too), "
                                      "same GPU"}}
        del t_in
        if kb == 4 and not has_v and key_bits == 32:
            lib["cub.DeviceRadixSort.SortKeys"] = cub_context(d_keys, n, stream)

    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        n_sample = n
        rate, secs = cpu_oracle_rate(wl, n_sample)
        cpu = {"value": rate, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle sort of {n_sample} keys of the same workload ({secs:.1f} s), "
                         f"single thread of {os.cpu_count()} host cores"}

    # the metric's second half: batched and served sorts against plain ones
    # (one GPU; every rank would measure the same thing again)
    batched = served = None
    if args.batched_served and wl == "radix_u32_100m" and world == 1 and not args.n:
        del ws, hbufs, houts, houtv, d_keys, d_out, d_vals, d_outv
        torch.cuda.empty_cache()
        batched = batched_summary(dev, steps=max(3, min(args.steps, 5)), warmup=3)
        torch.cuda.empty_cache()
        served = served_summary(dev, rates=SUMMARY_RATES, count=1000)
        torch.cuda.empty_cache()

    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(wl), "data": "synthetic",
        "config": {"workload": desc, "n": n, "key_bits": key_bits, "parallelism": f"replicas x{world}",
                   "kernel_shape": ({"digit_bits": tuned[0], "block_threads": tuned[1], "items_per_thread": tuned[2],
                                     "chosen_by": "autotuner"} if algo == "radix" and tuned else None),
                   "l2": "inputs larger than L2 (%d MB keys vs 129 MB L2), no flush" % (n * kb // 2**20)},
        "clocks": clocks, "gpu_launches": launches, "roofline": roofline, "whole_sort": whole,
        "e2e": {"value": e2e_value, "unit": "Gkeys/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "rs_sort_host_u32/u64 or bs_sort_host_u32/u64 (host arrays in and out, one call per step)",
                "mode": "pipelined: calls round-robin over 3 streams with their own device buffers, so one call's "
                        "copies overlap another's sort",
                "serial_value": e2e_serial, "steps": e2e_steps,
                "repeats_ms": {"pipelined": pipe_all, "serial": serial_all},
                "timing": f"median of {E2E_REPEATS} repeats of {e2e_steps} steps each (the host link is shared "
                          "with other work on the machine)",
                "link": dict(link, bound_value=link_bound(n, h2d, d2h, ms / args.steps, link),
                             note="bound_value: the pipelined ceiling set by the sort time and the host link's "
                                  "measured copy rates on these pinned buffers")},
        "cpu_baseline": cpu, "context": lib, "batched": batched, "served": served,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ batched and served, for the default line
SUMMARY_RATES = (2_000, 5_000, 20_000)


def batched_summary(dev, steps=5, warmup=3):
    """The batched workload (20,000 uint32 arrays, sizes log-uniform in
    [256, 2,000,000], seed 0, ~4.4e9 keys) sorted by one CUDA-graph launch of
    the segmented sort (autotuned pass shape) against one rs_sort_u32 call
    per array on the same stream.  Latency of an array: from the moment all
    arrays are handed over to its completion (plain: the event after its own
    sort; batched: the end of the graph)."""
    import numpy as np
    import torch

    import paper_1206_3511_gb300 as rs

    count = WORKLOADS["batched_u32_20k"][3]
    sizes, off, d_keys = batched_inputs(count, 0, dev)
    n_total = int(off[-1])
    d_out = torch.empty_like(d_keys)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    plan = rs.Plan(rs.RS_PLAN_SEGMENTED, d_keys, d_out, seg_offsets=d_off, autotune=True)
    seg_shape, graph_kernels, _ = plan.info()
    for _ in range(warmup):
        plan.launch(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / steps
    if rs.get_status(plan.ws):
        raise rs.SortError(rs.get_status(plan.ws), "batched device status")
    for i in (0, count // 2, count - 1):  # spot check (the tests hold the oracle checks)
        a, b = int(off[i]), int(off[i + 1])
        assert np.array_equal(d_out[a:b].cpu().numpy().view(np.uint32),
                              np.sort(d_keys[a:b].cpu().numpy().view(np.uint32))), f"batched array {i} wrong"
    ws_plain = rs.workspace(rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, 4, False, int(sizes.max()), 32, 0, 0), dev)
    kp, op = d_keys.data_ptr(), d_out.data_ptr()
    offs = [int(x) for x in off]

    def plain_step(events=None):
        for i in range(count):
            a, b = offs[i], offs[i + 1]
            rc = rs.rs_sort_u32(kp + 4 * a, op + 4 * a, None, None, b - a, 32, ws_plain, ws_plain.numel(), stream)
            if rc:
                raise rs.SortError(rc, "plain sort")
            if events is not None:
                events[i].record(stream)

    plain_step()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(count)]
    plain_ms = []
    for _ in range(2):
        s0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        plain_step(evs)
        torch.cuda.synchronize()
        plain_ms.append(s0.elapsed_time(evs[-1]))
    plain_lat = [s0.elapsed_time(e) for e in evs]
    clocks = sampler.stop()
    plan.close()
    del plan, d_keys, d_out, ws_plain
    plain_t = float(np.median(plain_ms))
    return {
        "workload": WORKLOADS["batched_u32_20k"][6], "arrays": count, "keys": n_total,
        "graph": {"gkeys_s": n_total / (graph_ms / 1e3) / 1e9, "ms_per_batch": graph_ms, "steps": steps,
                  "p50_ms": graph_ms, "p99_ms": graph_ms, "kernel_nodes": graph_kernels,
                  "pass_shape": {"block_threads": seg_shape[1], "items_per_thread": seg_shape[2]}},
        "plain": {"gkeys_s": n_total / (plain_t / 1e3) / 1e9, "ms_per_batch": plain_t, "steps": len(plain_ms),
                  "p50_ms": _pct(plain_lat, 50), "p99_ms": _pct(plain_lat, 99),
                  "note": "one rs_sort_u32 call per array, in order, one stream, one workspace"},
        "speedup": plain_t / graph_ms, "clocks": clocks,
        "timing": "CUDA events on the launch stream; inputs (17.5 GB) larger than L2, no flush",
    }


def served_summary(dev, rates=SUMMARY_RATES, count=1000):
    """The served mix (Poisson arrivals; sizes log-uniform in [1e3, 5e7]
    keys; 70% uint32 keys only, 30% uint64 keys + uint32 values;
    distributions 0-6 drawn per request; radix requests) through the sort
    server (4 streams, continuous batching) against a plain loop that calls
    rs_sort_u32/u64 once per request at its arrival, on one stream.  Latency:
    scheduled arrival to completion seen on the host (the server's
    completion record; for the plain loop, a host thread that waits on each
    request's event in order).  Inputs are resident on the device before the
    clock starts; the served keys per run are ~4.6e9."""
    import numpy as np
    import torch

    import paper_1206_3511_gb300 as rs
    import synth
    from paper_1206_3511_gb300 import _lib

    sizes, kinds, dists = synth.served_mix(count, SERVED_LO, SERVED_HI, seed=0)
    big = int(sizes.max())
    src_k = {}
    for d in sorted(set(dists.tolist())):
        if np.any((dists == d) & (kinds == 0)):
            src_k[(0, d)] = synth.keys_u32_torch(big, d, seed=0, device=dev)
        if np.any((dists == d) & (kinds == 1)):
            src_k[(1, d)] = synth.keys_u64_shaped_torch(big, d, seed=0, device=dev)
    src_v = torch.arange(big, dtype=torch.int32, device=dev)
    ARENA = 60 * 10**9
    arena = torch.empty(ARENA, dtype=torch.uint8, device=dev)
    abase = arena.data_ptr()
    out_off, out_end, lap = [], [], []
    head, cur_lap = 0, 0
    for i in range(count):
        nb_out = (int(sizes[i]) * (4 if kinds[i] == 0 else 12) + 255) // 256 * 256
        if head + nb_out > ARENA:
            head, cur_lap = 0, cur_lap + 1
        out_off.append(head)
        out_end.append(head + nb_out)
        lap.append(cur_lap)
        head += nb_out
    reqs = []
    for i in range(count):
        n, kd, d = int(sizes[i]), int(kinds[i]), int(dists[i])
        kb = 4 if kd == 0 else 8
        kin, kout = src_k[(kd, d)].data_ptr(), abase + out_off[i]
        vin = src_v.data_ptr() if kd == 1 else None
        vout = abase + out_off[i] + 8 * n if kd == 1 else None
        reqs.append(_lib.RsRequest(rs.RS_ALGO_RADIX, kb, kin, kout, vin, vout, n, 8 * kb, 1, 0, 0))
    total_keys = int(sizes.sum())

    def must_wait_for(j, i):  # request j's output region is reused by request i
        return lap[j] < lap[i] - 1 or (lap[j] == lap[i] - 1 and out_off[j] < out_end[i])

    def run_server(rate, seed):
        srv = rs.Server(SERVED_BUDGET, SERVED_BUDGET, num_streams=4, max_batch=64, device=dev)
        arr = synth.poisson_arrivals(count, rate, seed=seed) * 1e3
        tickets, oldest = [0] * count, 0
        t0 = time.monotonic() * 1e3 + 2.0
        for i in range(count):
            while oldest < i and must_wait_for(oldest, i):
                srv.wait(tickets[oldest])
                oldest += 1
            while time.monotonic() * 1e3 < t0 + arr[i]:
                pass
            rc, tickets[i] = _lib.rs_server_submit(srv.handle, reqs[i])
            if rc:
                raise rs.SortError(rc, "submit")
        lat, done = [], []
        for i in range(count):
            rc = srv.wait(tickets[i])
            if rc:
                raise rs.SortError(rc, f"served request {i}")
            _, r = srv.result(tickets[i])
            done.append(r.t_done_ms)
            lat.append(r.t_done_ms - (t0 + arr[i]))
            srv.release(tickets[i])
        st = srv.stats()
        srv.close()
        span = max(done) - t0
        return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "gkeys_s": total_keys / (span / 1e3) / 1e9,
                "batches": int(st.batches), "batched_requests": int(st.batched_requests),
                "max_queued": int(st.max_queued)}

    ws_bytes = max(rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, 4, False, big, 32, 0, 0),
                   rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, 8, True, big, 64, 0, 0))
    ws = rs.workspace(ws_bytes, dev)
    pstream = torch.cuda.Stream(device=dev)

    def run_plain(rate, seed):
        """One rs_sort_* call per request at its arrival, in order, on one
        stream with one workspace; a host thread stamps each completion."""
        arr = synth.poisson_arrivals(count, rate, seed=seed) * 1e3
        evs = [torch.cuda.Event() for _ in range(count)]
        issued = [threading.Event() for _ in range(count)]
        done = [0.0] * count

        def poll():
            for i in range(count):
                issued[i].wait()
                while not evs[i].query():
                    time.sleep(20e-6)
                done[i] = time.monotonic() * 1e3

        th = threading.Thread(target=poll)
        th.start()
        t0 = time.monotonic() * 1e3 + 2.0
        for i in range(count):
            q = reqs[i]
            while time.monotonic() * 1e3 < t0 + arr[i]:
                pass
            fn = rs.rs_sort_u32 if q.key_bytes == 4 else rs.rs_sort_u64
            rc = fn(q.keys_in, q.keys_out, q.vals_in, q.vals_out, q.n, q.key_bits, ws, ws_bytes, pstream)
            if rc:
                raise rs.SortError(rc, f"plain request {i}")
            evs[i].record(pstream)
            issued[i].set()
        th.join()
        lat = [done[i] - (t0 + arr[i]) for i in range(count)]
        span = max(done) - t0
        return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "gkeys_s": total_keys / (span / 1e3) / 1e9}

    run_server(1e6, 99)  # warm-up
    run_plain(1e6, 99)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sampler.start()
    rows = []
    for j, rate in enumerate(rates):
        rows.append({"rate_per_s": rate, "server": run_server(rate, j), "plain": run_plain(rate, j)})
    clocks = sampler.stop()
    if rs.get_status(ws):
        raise rs.SortError(rs.get_status(ws), "plain served device status")
    # spot check: the last uint32 request below 2M keys whose region is not reused
    for i in range(count - 1, -1, -1):
        n, kd, d = int(sizes[i]), int(kinds[i]), int(dists[i])
        if kd != 0 or n > 2_000_000 or any(out_off[j] < out_end[i] and out_off[i] < out_end[j]
                                           for j in range(i + 1, count)):
            continue
        got = arena[out_off[i]: out_off[i] + 4 * n].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, np.sort(src_k[(0, d)][:n].cpu().numpy().view(np.uint32))), "served output wrong"
        break
    del arena, src_k, src_v, ws
    return {
        "workload": WORKLOADS["served_mix"][6].replace("vs a FIFO of one sort per request on one stream",
                                                        "radix requests"),
        "requests_per_rate": count, "keys_per_run": total_keys, "budget_bytes": SERVED_BUDGET,
        "server": "rs_server: 4 streams, continuous batching of up to 64 requests of <= 262,144 keys",
        "plain": "one rs_sort_u32/u64 call per request at its arrival, one stream, one workspace",
        "rates": rows, "clocks": clocks,
    }


# ------------------------------------------------------------------ batched (segmented) workload
def _roofline_from_stats(kstats, steps, step_bytes_of, hbm_peak, peak_src, traffic=None):
    """Roofline of the kernel with the most device time: its algorithmic
    bytes per step (step_bytes_of(name, launches per step)) over its time per
    step."""
    if not kstats:
        return None
    top = max(kstats, key=lambda k: kstats[k][1])
    nl, tot = kstats[top]
    per_step = nl / steps
    step_bytes = step_bytes_of(top, per_step)
    achieved = step_bytes / (tot / steps / 1e3) / 1e9
    return {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": f"{peak_src} copy bandwidth",
            "algorithmic_bytes_per_launch": step_bytes / per_step, "avg_launch_ms": tot / nl, "launches": nl}


def _pct(xs, q):
    import numpy as np

    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def batched_inputs(count, rank, dev, lo=BATCH_LO, hi=BATCH_HI):
    import numpy as np

    import synth

    sizes = synth.log_uniform_sizes(count, lo, hi, seed=0)
    off = synth.segment_offsets(sizes)
    n_total = int(off[-1])
    keys = synth.u32_torch(n_total, seed=rank, dist_id=0, device=dev)
    return sizes, off, keys


def run_batched(args):
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
    count = args.n or WORKLOADS[wl][3]
    sizes, off, d_keys = batched_inputs(count, rank, dev, *BATCH_SIZES[wl])
    n_total = int(off[-1])
    d_out = torch.empty_like(d_keys)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    # the plan's autotuner times every compiled pass shape on this batch and
    # captures the fastest into the graph
    plan = rs.Plan(rs.RS_PLAN_SEGMENTED, d_keys, d_out, seg_offsets=d_off, autotune=True)
    seg_shape, graph_kernels, _ = plan.info()

    sampler = ClockSampler(dev)
    sampler.start()
    for _ in range(max(3, args.warmup)):
        plan.launch(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.launch(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    status = rs.get_status(plan.ws)
    if status:
        raise rs.SortError(status, "device status after the timed steps")

    # per-kernel times: graph replays record no events, so the same sort runs
    # as eager calls with event profiling
    prof_steps = 3
    seg_ws = plan.ws
    rs.rs_profile_enable(True)
    launches0 = rs.rs_launch_count()
    for _ in range(prof_steps):
        rs.check(rs.rs_sort_segmented_u32_ex(d_keys, d_out, None, None, d_off, count, n_total, 32, seg_ws,
                                             seg_ws.numel(), stream, seg_shape), "segmented")
    torch.cuda.synchronize()
    launches_per_step = (rs.rs_launch_count() - launches0) / prof_steps
    rs.rs_profile_enable(False)
    kstats = rs.rs_profile_read()

    # spot check: a few arrays against a host sort (the tests hold the oracle checks)
    for i in (0, count // 2, count - 1):
        a, b = int(off[i]), int(off[i + 1])
        got = d_out[a:b].cpu().numpy().view(np.uint32)
        want = np.sort(d_keys[a:b].cpu().numpy().view(np.uint32), kind="stable")
        assert np.array_equal(got, want), f"batched output wrong in array {i}"

    # one rs_sort_u32 call per array (the plain path), same stream, one workspace
    big = int(sizes.max())
    ws_plain = rs.workspace(rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, 4, False, big, 32, 0, 0), d_keys.device)
    kp, op = d_keys.data_ptr(), d_out.data_ptr()
    offs = [int(x) for x in off]

    def plain_step(events=None):
        for i in range(count):
            a, b = offs[i], offs[i + 1]
            rc = rs.rs_sort_u32(kp + 4 * a, op + 4 * a, None, None, b - a, 32, ws_plain, ws_plain.numel(), stream)
            if rc:
                raise rs.SortError(rc, "plain sort")
            if events is not None:
                events[i].record(stream)

    plain_step()
    torch.cuda.synchronize()
    plain_steps = max(1, min(args.steps, 3))
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(plain_steps):
        plain_step()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1) / plain_steps
    # completion latency of every array when all are handed over at once:
    # plain = the event after its own sort; batched = the end of the graph
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(count)]
    s0 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    plain_step(evs)
    torch.cuda.synchronize()
    plain_lat = [s0.elapsed_time(e) for e in evs]
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    plan.launch(stream)
    g1.record(stream)
    torch.cuda.synchronize()
    batched_lat = g0.elapsed_time(g1)

    # end to end through the host-buffer segmented call
    # (rs_sort_segmented_host_u32): pinned host keys and offsets in, sorted
    # keys out, one library call copying in, sorting with the tuned shape and
    # copying out.  Serial: the whole batch in one call per step.
    h_keys = torch.empty(n_total, dtype=torch.int32, pin_memory=True)
    h_keys.copy_(d_keys)
    h_out = torch.empty_like(h_keys, pin_memory=True)
    h_off = torch.from_numpy(off.view(np.int64)).pin_memory()
    e2e_steps = max(3, min(args.steps, 5))
    hbytes = rs.rs_segmented_host_bytes(4, 0, n_total, count, 32)
    hbuf = rs.workspace(hbytes, d_keys.device)

    def host_batch(strm):
        rs.check(rs.rs_sort_segmented_host_u32(h_keys, h_out, None, None, h_off, count, n_total, 32, hbuf, hbytes,
                                               strm, seg_shape), "segmented host-buffer sort")

    host_batch(stream)
    torch.cuda.synchronize()

    def serial_run():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            host_batch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    serial_all = [serial_run() for _ in range(E2E_REPEATS)]
    e2e_serial_ms = float(np.median(serial_all))
    assert rs.get_status(hbuf) == 0
    del hbuf

    # Pipelined end to end: the batch in G groups of consecutive arrays, one
    # host-buffer call per group, the calls round-robin over three streams
    # with their own device buffers, so that one group's copies overlap other
    # groups' sorts.
    G, S = 8, 3
    bounds = [int(x) for x in np.linspace(0, count, G + 1).round()]
    groups = []
    for g in range(G):
        a, b = bounds[g], bounds[g + 1]
        if b <= a:
            continue
        k0, k1 = int(off[a]), int(off[b])
        goff = torch.from_numpy((off[a:b + 1] - off[a]).view(np.int64)).pin_memory()
        groups.append((a, b, k0, k1, goff))
    gbytes = max(rs.rs_segmented_host_bytes(4, 0, k1 - k0, b - a, 32) for a, b, k0, k1, _ in groups)
    gbufs = [rs.workspace(gbytes, d_keys.device) for _ in range(S)]
    gstreams = [torch.cuda.Stream() for _ in range(S)]
    calls = [0]  # the rotation over the streams continues across steps

    def pipe_step():
        for a, b, k0, k1, goff in groups:
            j = calls[0] % S
            calls[0] += 1
            rs.check(rs.rs_sort_segmented_host_u32(h_keys[k0:k1], h_out[k0:k1], None, None, goff, b - a, k1 - k0,
                                                   32, gbufs[j], gbytes, gstreams[j], seg_shape),
                     "segmented host-buffer group")

    pipe_step()
    torch.cuda.synchronize()

    def pipe_run():
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for gs in gstreams:
            gs.wait_event(p0)
        for _ in range(e2e_steps):
            pipe_step()
        for gs in gstreams:
            done = torch.cuda.Event()
            done.record(gs)
            stream.wait_event(done)
        p1.record(stream)
        torch.cuda.synchronize()
        return p0.elapsed_time(p1)

    pipe_all = [pipe_run() for _ in range(E2E_REPEATS)]
    e2e_ms = float(np.median(pipe_all))
    for j in range(S):
        assert rs.get_status(gbufs[j]) == 0
    for i in (0, count // 2, count - 1):  # the downloaded result, spot-checked
        a, b = int(off[i]), int(off[i + 1])
        assert torch.equal(h_out[a:b], d_out[a:b].cpu()), f"pipelined result wrong in array {i}"
    link = host_link_rates(h_keys, h_out, d_out, d_keys)  # overwrites the start of h_out and d_out

    ms, e2e_ms, e2e_serial_ms, plain_ms = max_over_ranks([ms, e2e_ms, e2e_serial_ms, plain_ms], device=dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    value = job_rate(n_total * args.steps, world, ms)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    n_large = int(sizes[sizes > 4096].sum())
    n_small = n_total - n_large

    n_tiny = int(sizes[sizes <= 256].sum())

    def step_bytes_of(name, per_step):
        if name == "onesweep_seg_pass":
            return 2 * n_large * 4 * per_step
        if name == "local_sort":
            return 2 * (n_small - n_tiny) * 4
        if name == "tiny_sort":
            return 2 * n_tiny * 4
        return n_large * 4 * per_step

    roofline = _roofline_from_stats(kstats, prof_steps, step_bytes_of, hbm_peak, peak_src)
    if roofline and roofline["kernel"] == "onesweep_seg_pass" and wl == "batched_u32_20k" and \
            count == WORKLOADS[wl][3]:
        roofline["traffic"] = ncu_traffic("onesweep_seg_pass", wl)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = _batched_cpu_sample(sizes, off, d_keys)
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS[wl][6], "arrays": count, "n_total": n_total,
                   "parallelism": f"replicas x{world}",
                   "kernel_shape": {"digit_bits": seg_shape[0], "block_threads": seg_shape[1],
                                    "items_per_thread": seg_shape[2], "chosen_by": "autotuner"},
                   "l2": "inputs larger than L2 (%d MB keys vs 129 MB L2), no flush" % (n_total * 4 // 2**20)},
        "clocks": clocks, "gpu_launches": graph_kernels * args.steps, "graph_kernel_nodes": graph_kernels,
        "eager_launches_per_step": launches_per_step,
        "roofline": roofline,
        "batched": {"ms_per_step": ms / args.steps, "p50_ms": batched_lat, "p99_ms": batched_lat,
                    "host_launches_per_step": 1},
        "plain": {"value": n_total / (plain_ms / 1e3) / 1e9, "unit": "Gkeys/s", "ms_per_step": plain_ms,
                  "p50_ms": _pct(plain_lat, 50), "p99_ms": _pct(plain_lat, 99), "host_calls_per_step": count,
                  "steps": plain_steps},
        "latency_note": "completion time of each array after all arrays are handed over at once",
        "kernels": {k: {"launches": v[0], "avg_ms": v[1] / v[0]} for k, v in kstats.items()},
        "e2e": {"value": job_rate(n_total * e2e_steps, world, e2e_ms), "unit": "Gkeys/s",
                "h2d_bytes_per_step": n_total * 4, "d2h_bytes_per_step": n_total * 4,
                "api": "rs_sort_segmented_host_u32 (host arrays and offsets in, sorted keys out)",
                "mode": "pipelined: the batch in 8 groups of consecutive arrays, one call per group, the calls "
                        "round-robin over 3 streams with their own device buffers",
                "serial_value": job_rate(n_total * e2e_steps, world, e2e_serial_ms), "steps": e2e_steps,
                "repeats_ms": {"pipelined": pipe_all, "serial": serial_all},
                "timing": f"median of {E2E_REPEATS} repeats of {e2e_steps} steps each (the host link is shared "
                          "with other work on the machine)",
                "link": dict(link, bound_value=link_bound(n_total, 4 * n_total, 4 * n_total, ms / args.steps, link),
                             note="bound_value: the pipelined ceiling set by the sort time and the host link's "
                                  "measured copy rates on these pinned buffers")},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _batched_cpu_sample(sizes, off, d_keys=None, budget_keys=150_000_000):
    """The oracle's segmented sort of the first arrays of the batch, up to
    about budget_keys keys: (Gkeys/s, ...)."""
    import numpy as np

    import oracle
    import synth

    oracle.build()
    m = int(np.searchsorted(np.cumsum(sizes), budget_keys)) + 1
    m = min(m, sizes.size)
    sub = synth.segment_offsets(sizes[:m])
    n = int(sub[-1])
    if d_keys is not None:
        keys = d_keys[:n].cpu().numpy().view(np.uint32)
    else:
        keys = synth.u32(n, 0, 0)
    t0 = time.perf_counter()
    oracle.segmented_radix_sort(keys, sub, None, 32)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "sample_keys": n,
            "sample": f"oracle segmented sort of the first {m} arrays of the batch ({n} keys, {dt:.1f} s), "
                      f"single thread of {os.cpu_count()} host cores"}


# ------------------------------------------------------------------ the paper's cases
def run_paper_cases(args):
    """The paper's Table 1 grid on the GPU: six input cases at three sizes,
    radix and bucket sort, with the workspace each call needs (the analogue
    of Table 2).  Keys are copied to the device before timing."""
    import numpy as np
    import torch

    import paper_1206_3511_gb300 as rs
    import synth

    world, rank, local = _dist_env()
    torch.cuda.set_device(local if world > 1 else 0)
    rs.load()
    sizes = (10**6, 10**7, 10**8) if not args.n else (args.n,)
    steps = max(3, min(args.steps, 20))
    stream = torch.cuda.current_stream()
    rows = []
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    launches0 = rs.rs_launch_count()
    for case, (desc, M) in synth.PAPER_CASES.items():
        for si, n in enumerate(sizes):
            keys = synth.paper_case_keys(n, case, seed=rank)
            d_keys = torch.from_numpy(keys.view(np.int32)).cuda()
            d_out = torch.empty_like(d_keys)
            key_bits = max(1, int(M - 1).bit_length())
            nb = max(1, n // 16)
            ws_r = rs.rs_workspace_bytes(rs.RS_ALGO_RADIX, 4, False, n, key_bits, 0, 0)
            ws_b = rs.rs_workspace_bytes(rs.RS_ALGO_BUCKET, 4, False, n, 0, nb, 0)
            ws = rs.workspace(max(ws_r, ws_b), d_keys.device)
            calls = {
                "radix": lambda: rs.rs_sort_u32(d_keys, d_out, None, None, n, key_bits, ws, ws.numel(), stream),
                "bucket": lambda: rs.bs_sort_u32(d_keys, d_out, None, None, n, 0, M - 1, nb, ws, ws.numel(), stream),
            }
            row = {"case": case, "input": desc, "n": n, "key_bits": key_bits, "num_buckets": nb,
                   "workspace_mb": {"radix": ws_r / 2**20, "bucket": ws_b / 2**20}, "input_mb": n * 4 / 2**20}
            want = np.sort(keys)
            for algo, fn in calls.items():
                for _ in range(max(3, args.warmup)):
                    rs.check(fn(), algo)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    rs.check(fn(), algo)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                if rs.get_status(ws):
                    raise rs.SortError(rs.get_status(ws), algo)
                assert np.array_equal(d_out.cpu().numpy().view(np.uint32), want), f"{algo} case {case} n={n}"
                paper_s = PAPER_TABLE1_S[case][si + (3 if algo == "bucket" else 0)] if n in (10**6, 10**7, 10**8) else None
                row[algo] = {"ms": ms, "gkeys_s": n / (ms / 1e3) / 1e9, "paper_laptop_s": paper_s}
            rows.append(row)
            del d_keys, d_out, ws
    clocks = sampler.stop()
    launches = rs.rs_launch_count() - launches0
    if rank != 0:
        return
    top = [r for r in rows if r["case"] == 1 and r["n"] == max(sizes)][0]
    print(json.dumps({
        "metric": METRIC, "value": top["radix"]["gkeys_s"], "unit": "Gkeys/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": top["radix"]["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS["paper_cases"][6], "sizes": list(sizes),
                   "l2": "every size is timed as is; 10^6 and 10^7 fit in L2 (context rows)"},
        "value_note": "radix sort of case 1 at the largest size", "clocks": clocks, "gpu_launches": launches,
        "roofline": None, "cases": rows,
        "paper_note": "paper_laptop_s: the paper's Table 1 (sequential C++, Intel i5 laptop), context only",
        "e2e": None, "cpu_baseline": None}), flush=True)


# ------------------------------------------------------------------ served workload
def served_bytes(n, kind):
    """Algorithmic HBM bytes of one radix request of the served mix: kind 0
    is uint32 keys only, kind 1 uint64 keys with uint32 values."""
    return sort_bytes("radix", n, 4, False) if kind == 0 else sort_bytes("radix", n, 8, True)


def run_served(args):
    import ctypes

    import numpy as np
    import torch

    import paper_1206_3511_gb300 as rs
    import synth
    from paper_1206_3511_gb300 import _lib

    world, rank, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    rs.load()
    count = args.n or WORKLOADS["served_mix"][3]
    rates = SERVED_RATES if not args.rates else tuple(int(r) for r in args.rates.split(","))
    sizes, kinds, dists = synth.served_mix(count, SERVED_LO, SERVED_HI, seed=rank)
    big = int(sizes.max())
    # resident inputs: one array per (kind, distribution); request i reads a prefix
    src_k, src_v = {}, None
    for d in sorted(set(dists.tolist())):  # built on the device (same bits as the numpy forms)
        if np.any((dists == d) & (kinds == 0)):
            src_k[(0, d)] = synth.keys_u32_torch(big, d, seed=rank, device=dev)
        if np.any((dists == d) & (kinds == 1)):
            src_k[(1, d)] = synth.keys_u64_shaped_torch(big, d, seed=rank, device=dev)
    if np.any(kinds == 1):
        src_v = torch.arange(big, dtype=torch.int32, device=dev)
    # outputs: a circular arena; request i's keys (and values) go at the head,
    # and before a region is reused the requests that held it are waited for
    ARENA = 60 * 10**9
    arena = torch.empty(ARENA, dtype=torch.uint8, device=dev)
    abase = arena.data_ptr()
    out_off, out_end, lap = [], [], []
    head, cur_lap = 0, 0
    for i in range(count):
        nb_out = int(sizes[i]) * (4 if kinds[i] == 0 else 12)
        nb_out = (nb_out + 255) // 256 * 256
        if head + nb_out > ARENA:
            head, cur_lap = 0, cur_lap + 1
        out_off.append(head)
        out_end.append(head + nb_out)
        lap.append(cur_lap)
        head += nb_out
    def build_requests(bucket_share):
        """One request per draw; a share of them (drawn) use the bucket sort
        with the distribution's declared bounds and n/16 buckets."""
        use_bucket = synth.unit_doubles(count, rank, 45) < bucket_share
        reqs, nbytes = [], 0
        for i in range(count):
            n, kd, d = int(sizes[i]), int(kinds[i]), int(dists[i])
            lo, hi = synth.DECLARED_BOUNDS[d]
            kb = 4 if kd == 0 else 8
            if kd == 1:
                lo, hi = lo << 32, (hi << 32) | 0xFFFFFFFF
            kin, kout = src_k[(kd, d)].data_ptr(), abase + out_off[i]
            vin = src_v.data_ptr() if kd == 1 else None
            vout = abase + out_off[i] + 8 * n if kd == 1 else None
            if use_bucket[i]:
                reqs.append(_lib.RsRequest(rs.RS_ALGO_BUCKET, kb, kin, kout, vin, vout, n, 0, lo, hi, 0))
                nbytes += sort_bytes("bucket", n, kb, kd == 1)
            else:
                reqs.append(_lib.RsRequest(rs.RS_ALGO_RADIX, kb, kin, kout, vin, vout, n, 8 * kb, 1, 0, 0))
                nbytes += served_bytes(n, kd)
        return reqs, nbytes, int(use_bucket.sum())

    total_keys = int(sizes.sum())
    reqs, total_bytes, _ = build_requests(0.0)

    def run_mode(rate, num_streams, max_batch, seed):
        srv = rs.Server(SERVED_BUDGET, SERVED_BUDGET, num_streams=num_streams, max_batch=max_batch, device=dev)
        arr = synth.poisson_arrivals(count, rate, seed=seed) * 1e3  # ms
        tickets = [0] * count
        lag = []
        oldest = 0  # requests below this index no longer hold arena space
        t0 = time.monotonic() * 1e3 + 2.0
        for i in range(count):
            # wait for the earlier requests whose output region this one
            # reuses: every request two laps back, and those of the previous
            # lap that start before this region ends
            while oldest < i and (lap[oldest] < lap[i] - 1 or
                                  (lap[oldest] == lap[i] - 1 and out_off[oldest] < out_end[i])):
                srv.wait(tickets[oldest])
                oldest += 1
            target = t0 + arr[i]
            while time.monotonic() * 1e3 < target:
                pass
            lag.append(time.monotonic() * 1e3 - target)
            rc, tickets[i] = _lib.rs_server_submit(srv.handle, reqs[i])
            if rc:
                raise rs.SortError(rc, "submit")
        lat, done = [], []
        for i in range(count):
            rc = srv.wait(tickets[i])
            if rc:
                raise rs.SortError(rc, f"request {i}")
            _, r = srv.result(tickets[i])
            done.append(r.t_done_ms)
            lat.append(r.t_done_ms - (t0 + arr[i]))
            srv.release(tickets[i])
        st = srv.stats()
        srv.close()
        span_ms = max(done) - t0
        return {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "max_ms": max(lat),
                "gkeys_s": total_keys / (span_ms / 1e3) / 1e9, "span_ms": span_ms,
                "offered_gkeys_s": total_keys / (arr[-1] / 1e3) / 1e9,
                "submit_lag_p99_ms": _pct(lag, 99), "submitted": int(st.submitted),
                "admitted": int(st.submitted - st.rejected), "rejected": int(st.rejected),
                "completed": int(st.completed), "batches": int(st.batches),
                "batched_requests": int(st.batched_requests), "max_queued": int(st.max_queued),
                "max_in_use_gb": st.max_in_use_bytes / 1e9}

    def knee(rows, mode):
        """The highest rate whose p99 stays within 4x the p99 at the lowest rate."""
        base = rows[0][mode]["p99_ms"]
        ok = [r["rate_per_s"] for r in rows if r[mode]["p99_ms"] <= 4 * base]
        return max(ok) if ok else None

    # warm-up: every request once through the server
    for _ in range(max(1, min(args.warmup, 2))):
        run_mode(1e6, 4, 64, seed=99)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sampler.start()
    launches0 = rs.rs_launch_count()
    sweep = []
    for j, rate in enumerate(rates):
        srv_res = run_mode(rate, 4, 64, seed=j)
        fifo_res = run_mode(rate, 1, 1, seed=j)
        sweep.append({"rate_per_s": rate, "server": srv_res, "fifo": fifo_res})
    radix_reqs, radix_bytes = reqs, total_bytes
    sweep_bucket = []
    if args.bucket_sweep:
        reqs, bucket_bytes, n_bucket = build_requests(0.5)
        for j, rate in enumerate(rates):
            sweep_bucket.append({"rate_per_s": rate, "server": run_mode(rate, 4, 64, seed=j),
                                 "fifo": run_mode(rate, 1, 1, seed=j)})
        reqs = radix_reqs
    launches = rs.rs_launch_count() - launches0
    clocks = sampler.stop()
    torch.cuda.synchronize()
    # replicas: every rank serves its own copy of the mix; the job's time at
    # the top rate is the slowest rank's
    top_span = max_over_ranks([sweep[-1]["server"]["span_ms"]], device=dev)[0]

    # spot check: the last small requests of the last run (their output
    # regions are not reused after them), against a host sort
    checked = 0
    for i in range(count - 1, -1, -1):
        n, kd, d = int(sizes[i]), int(kinds[i]), int(dists[i])
        if n > 2_000_000 or any(out_off[j] < out_end[i] and out_off[i] < out_end[j] for j in range(i + 1, count)):
            continue
        o = out_off[i]
        if kd == 0:
            inp = src_k[(0, d)][:n].cpu().numpy().view(np.uint32)
            got = arena[o: o + 4 * n].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, np.sort(inp, kind="stable")), f"served request {i} wrong"
        else:
            inp = src_k[(1, d)][:n].cpu().numpy().view(np.uint64)
            order = np.argsort(inp, kind="stable")
            got_k = arena[o: o + 8 * n].cpu().numpy().view(np.uint64)
            got_v = arena[o + 8 * n: o + 12 * n].cpu().numpy().view(np.uint32)
            assert np.array_equal(got_k, inp[order]) and np.array_equal(got_v, order.astype(np.uint32)), \
                f"served request {i} wrong"
        checked += 1
        if checked == 4:
            break
    if rank != 0:
        return
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    peak_src = "measured" if peaks.get("hbm_gbs") else "fallback"
    top = sweep[-1]["server"]
    achieved = job_rate(radix_bytes, world, top_span)
    line = {
        "metric": METRIC, "value": job_rate(total_keys, world, top_span), "unit": "Gkeys/s", "n_gpus": world,
        "steps": len(rates), "warmup": args.warmup, "ms_per_step": top["span_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
        "config": {"workload": WORKLOADS["served_mix"][6], "requests_per_rate": count, "keys_per_run": total_keys,
                   "rates_per_s": list(rates), "budget_bytes": SERVED_BUDGET,
                   "server": "4 streams, batches of up to 64 requests of <= 262,144 keys",
                   "fifo": "same server with 1 stream and no batching",
                   "l2": "inputs resident in HBM (%.1f GB per run) larger than L2, no flush" % (total_bytes / 1e9)},
        "value_note": "server throughput at the highest arrival rate (keys / (last completion - first arrival))",
        "clocks": clocks, "gpu_launches": launches,
        "roofline": {"kernel": "all kernels of the served mix", "bound": "hbm", "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                     "peak_source": f"{peak_src} copy bandwidth",
                     "algorithmic_bytes_per_run": radix_bytes},
        "sweep": sweep, "knee_per_s": {"server": knee(sweep, "server"), "fifo": knee(sweep, "fifo")},
        "sweep_half_bucket": sweep_bucket,
        "knee_half_bucket_per_s": ({"server": knee(sweep_bucket, "server"), "fifo": knee(sweep_bucket, "fifo")}
                                   if sweep_bucket else None),
        "e2e": {"value": job_rate(total_keys, world, top_span), "unit": "Gkeys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0,
                "note": "host-submitted requests, completion seen on the host; keys resident on the device"},
        "cpu_baseline": None if args.no_cpu_baseline else _served_cpu_sample(sizes, kinds, dists),
    }
    print(json.dumps(line), flush=True)


def _served_cpu_sample(sizes, kinds, dists, budget_keys=100_000_000):
    """The oracle's radix sorts of the first requests of the mix, one after
    another, up to about budget_keys keys."""
    import numpy as np

    import oracle
    import synth

    oracle.build()
    done, t = 0, 0.0
    for i in range(sizes.size):
        n, kd, d = int(sizes[i]), int(kinds[i]), int(dists[i])
        if done and done + n > budget_keys:
            continue
        if kd == 0:
            keys, vals, kb = synth.keys_u32(n, d, seed=0), None, 32
        else:
            keys, vals, kb = synth.keys_u64_shaped(n, d, seed=0), synth.index_values(n), 64
        t0 = time.perf_counter()
        oracle.radix_sort(keys, vals, kb, 8)
        t += time.perf_counter() - t0
        done += n
        if done >= budget_keys:
            break
    return {"value": done / t / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "sample_keys": done,
            "sample": f"oracle radix sorts of {done} keys of the request mix, one after another ({t:.1f} s), "
                      f"single thread of {os.cpu_count()} host cores"}


def run_reference_batched(args):
    _, rank, _ = _dist_env()
    if rank != 0:
        return
    import synth

    count = args.n or WORKLOADS[args.workload][3]
    sizes = synth.log_uniform_sizes(count, *BATCH_SIZES[args.workload], seed=0)
    total_steps = max(1, args.warmup + args.steps)
    budget = max(5_000_000, 60 * 50_000_000 // total_steps)
    rates = []
    cpu = None
    for i in range(total_steps):
        cpu = _batched_cpu_sample(sizes, None, None, budget)
        if i >= args.warmup:
            rates.append(cpu["value"])
    value = statistics.median(rates)
    cpu["value"] = value
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cpu["sample_keys"] / value / 1e6,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload][6], "arrays": count, "parallelism": "none (1 CPU thread)"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def run_reference_served(args):
    _, rank, _ = _dist_env()
    if rank != 0:
        return
    import synth

    count = args.n or WORKLOADS["served_mix"][3]
    sizes, kinds, dists = synth.served_mix(count, SERVED_LO, SERVED_HI, seed=0)
    total_steps = max(1, args.warmup + args.steps)
    budget = max(5_000_000, 60 * 40_000_000 // total_steps)
    rates, cpu = [], None
    for i in range(total_steps):
        cpu = _served_cpu_sample(sizes, kinds, dists, budget)
        if i >= args.warmup:
            rates.append(cpu["value"])
    value = statistics.median(rates)
    cpu["value"] = value
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cpu["sample_keys"] / value / 1e6,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
        "config": {"workload": WORKLOADS["served_mix"][6], "parallelism": "none (1 CPU thread)"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse_args()
    kind = WORKLOADS[args.workload][0]
    if args.impl == "reference":
        if kind == "batched":
            run_reference_batched(args)
        elif kind == "served":
            run_reference_served(args)
        elif kind == "paper":
            print(json.dumps({"impl": "reference", "unavailable": "the paper-case grid is a report; its oracle "
                              "timings are the per-workload reference runs"}), flush=True)
        else:
            run_reference(args)
    elif kind == "paper":
        run_paper_cases(args)
    elif kind == "batched":
        run_batched(args)
    elif kind == "served":
        run_served(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
