"""The sort server: every request's result in the mix equals the result of
sorting it alone (zero tolerance), admission never exceeds the budget, small
requests are batched, requests that can never fit are refused, and shutdown
cancels what is still queued."""
import threading

import numpy as np
import pytest

import synth
from tests._util import assert_same, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _mix(seed=0, count=60):
    """Sizes log-uniform in [1000, 2000000], 70% u32 keys only, 30% u64 keys
    with index values, radix and bucket requests."""
    sizes = synth.log_uniform_sizes(count, 1000, 2_000_000, seed=seed, dist_id=31)
    kinds = synth.uniform_below(count, 10, seed, 32)
    algos = synth.uniform_below(count, 2, seed, 33)
    reqs = []
    for i, (n, k, a) in enumerate(zip(sizes.tolist(), kinds.tolist(), algos.tolist())):
        if k < 7:
            keys = synth.keys_u32(n, i % 7, seed=100 + i)
            vals = None
        else:
            keys = synth.keys_u64(n, 64, seed=100 + i)
            vals = synth.index_values(n)
        reqs.append((keys, vals, 1 if a else 0))
    return reqs


def _submit_all(rs, srv, reqs):
    """Stage every request on the device first, then submit them back to back
    (requests that arrive while others run are what gets batched)."""
    import torch

    staged = []
    for keys, vals, algo in reqs:
        kd = to_dev(keys)
        vd = to_dev(vals) if vals is not None else None
        ko = torch.empty_like(kd)
        vo = torch.empty_like(vd) if vd is not None else None
        staged.append((kd, ko, vd, vo, algo))
    torch.cuda.synchronize()
    handles = []
    for kd, ko, vd, vo, algo in staged:
        t = srv.submit(kd, ko, vd, vo, algo=algo)
        handles.append((t, ko, vo))
    return handles


def test_results_in_the_mix_equal_results_alone(rs, oracle):
    reqs = _mix(0, 60)
    with rs.Server(pool_bytes=6 << 30, num_streams=4, max_batch=16, batch_max_keys=1 << 18) as srv:
        handles = _submit_all(rs, srv, reqs)
        for (t, ko, vo), (keys, vals, algo) in zip(handles, reqs):
            assert srv.wait(t, 60_000) == 0
            gk = from_dev(ko, keys.dtype)
            if vals is None:
                assert_same(gk, oracle.radix_sort(keys), f"ticket {t}")
            else:
                wk, wv = oracle.radix_sort(keys, vals)
                assert_same(gk, wk, f"ticket {t} keys")
                assert_same(from_dev(vo, np.uint32), wv, f"ticket {t} values")
        st = srv.stats()
        assert st.completed == len(reqs) and st.rejected == 0
        assert st.batches >= 1 and st.batched_requests >= 2
        assert st.max_in_use_bytes <= st.budget_bytes


def test_budget_is_never_exceeded_and_everything_completes(rs):
    import torch

    budget = 300 << 20
    with rs.Server(pool_bytes=1 << 30, budget_bytes=budget, num_streams=4, max_batch=8) as srv:
        tickets = []
        outs = []
        for i in range(24):
            n = 3_000_000 if i % 3 == 0 else 100_000
            kd = to_dev(synth.u32(n, 60 + i, 0))
            ko = torch.empty_like(kd)
            tickets.append(srv.submit(kd, ko))
            outs.append((kd, ko))
        for t in tickets:
            assert srv.wait(t, 60_000) == 0
        st = srv.stats()
        assert st.completed == 24 and st.queued == 0
        assert 1 <= st.max_queued <= 24
        assert 0 < st.max_in_use_bytes <= budget
        for kd, ko in outs:
            a = ko.cpu().numpy().view(np.uint32)
            assert np.all(a[1:] >= a[:-1])


def test_submissions_from_many_threads(rs, oracle):
    import torch

    with rs.Server(pool_bytes=2 << 30, num_streams=3, max_batch=32) as srv:
        results = {}
        lock = threading.Lock()

        def worker(w):
            for j in range(10):
                keys = synth.u32(5000 + 977 * j + w, 70 + w * 10 + j, 0)
                kd = to_dev(keys)
                ko = torch.empty_like(kd)
                t = srv.submit(kd, ko)
                with lock:
                    results[t] = (keys, ko, kd)

        threads = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        for t, (keys, ko, _) in results.items():
            assert srv.wait(t, 60_000) == 0
            assert_same(from_dev(ko, np.uint32), np.sort(keys), f"thread ticket {t}")


def test_request_that_can_never_fit_is_refused(rs):
    import torch

    with rs.Server(pool_bytes=64 << 20, num_streams=2, max_batch=4) as srv:
        kd = torch.zeros(20_000_000, dtype=torch.int32, device="cuda")
        ko = torch.empty_like(kd)
        with pytest.raises(rs.SortError) as e:
            srv.submit(kd, ko)
        assert e.value.code == 4  # RS_ERR_BUDGET
        assert srv.stats().rejected == 1


def test_shutdown_cancels_queued_requests(rs):
    """With one stream and a budget that admits one request at a time, a
    cancelling shutdown returns without sorting the queue."""
    import time

    import torch

    keys = to_dev(synth.u32(8_000_000, 90, 0))
    outs = [torch.empty_like(keys) for _ in range(40)]
    torch.cuda.synchronize()
    srv = rs.Server(pool_bytes=512 << 20, budget_bytes=200 << 20, num_streams=1, max_batch=1)
    for ko in outs:
        srv.submit(keys, ko)
    st = srv.stats()
    assert st.submitted == 40 and st.queued >= 30
    assert st.queued <= st.max_queued <= 40
    t0 = time.perf_counter()
    assert rs.rs_server_destroy(srv.handle, True) == 0
    elapsed = time.perf_counter() - t0
    srv.handle = None
    torch.cuda.synchronize()
    # 40 sorts of 8M keys one after another take far longer than this
    assert elapsed < 0.5, elapsed


def test_released_requests_are_forgotten(rs):
    import torch

    keys = to_dev(synth.u32(10_000, 80, 0))
    out = torch.empty_like(keys)
    with rs.Server(pool_bytes=256 << 20, num_streams=2) as srv:
        t = srv.submit(keys, out)
        assert srv.wait(t, 60_000) == 0
        assert srv.release(t) == 0
        assert srv.release(t) == 1  # RS_ERR_INVALID_ARG: unknown ticket now
        rc, _ = srv.result(t)
        assert rc == 1


def test_large_unbatched_requests_in_the_mix_equal_results_alone(rs, oracle):
    """Requests above batch_max_keys run as single sorts beside the batched
    small ones: 12M and 10M u32 keys (radix; bucket over declared bounds),
    10M and 3M u64 keys with index values (radix; bucket over computed
    bounds), mixed with 24 small requests, each result compared with the
    oracle."""
    big = [
        (synth.keys_u32(12_000_000, 0, seed=201), None, 0, {}),
        (synth.keys_u32(10_000_000, 6, seed=202), None, 1, dict(zip(("min_key", "max_key"),
                                                                    synth.DECLARED_BOUNDS[6]))),
        (synth.keys_u64(10_000_000, 64, seed=203), synth.index_values(10_000_000), 0, {}),
        (synth.keys_u64(3_000_000, 40, seed=204), synth.index_values(3_000_000), 1, {}),
    ]
    small = [(synth.keys_u32(5000 + 311 * i, i % 7, seed=210 + i), None, 0, {}) for i in range(24)]
    reqs = big[:2] + small[:12] + big[2:] + small[12:]
    import torch

    with rs.Server(pool_bytes=8 << 30, num_streams=4, max_batch=16, batch_max_keys=1 << 18) as srv:
        handles = []
        for keys, vals, algo, bounds in reqs:
            kd = to_dev(keys)
            vd = to_dev(vals) if vals is not None else None
            ko = torch.empty_like(kd)
            vo = torch.empty_like(vd) if vd is not None else None
            torch.cuda.synchronize()
            handles.append((srv.submit(kd, ko, vd, vo, algo=algo, **bounds), ko, vo))
        for (t, ko, vo), (keys, vals, algo, _) in zip(handles, reqs):
            assert srv.wait(t, 120_000) == 0
            gk = from_dev(ko, keys.dtype)
            if vals is None:
                assert_same(gk, oracle.radix_sort(keys), f"ticket {t} n={keys.size}")
            else:
                wk, wv = oracle.radix_sort(keys, vals)
                assert_same(gk, wk, f"ticket {t} keys n={keys.size}")
                assert_same(from_dev(vo, np.uint32), wv, f"ticket {t} values n={keys.size}")
        assert srv.stats().completed == len(reqs)


@pytest.mark.parametrize("algo,n", [(0, 300_000), (0, 2000), (1, 300_000)])
def test_device_errors_reach_the_request(rs, algo, n):
    """A key above 2^key_bits (radix) or outside the declared bounds (bucket)
    is found on the device; the request must end with RS_ERR_KEY_RANGE, not
    RS_OK.  The 2,000-key radix request is sent with two good ones of the
    same type, so it may be batched; if it is, its batch reports the error
    too, and a good request that was not batched with it ends RS_OK."""
    import torch

    keys = synth.u32(n, 220 + n % 7, 0) >> np.uint32(8)  # 24-bit keys
    keys[n // 2] = 1 << 24 if algo == 0 else (1 << 24) + 5
    good = [synth.u32(n, 230 + j, 0) >> np.uint32(8) for j in range(2)]
    bounds = {} if algo == 0 else {"min_key": 0, "max_key": (1 << 24) - 1}
    with rs.Server(pool_bytes=1 << 30, num_streams=2, max_batch=8) as srv:
        outs, tickets = [], []
        for k in [keys] + good:
            kd = to_dev(k)
            ko = torch.empty_like(kd)
            torch.cuda.synchronize()
            tickets.append(srv.submit(kd, ko, algo=algo, key_bits=24 if algo == 0 else 0, **bounds))
            outs.append((k, ko))
        codes = [srv.wait(t, 60_000) for t in tickets]
        assert codes[0] == 3  # RS_ERR_KEY_RANGE
        batched = srv.stats().batches > 0
        for (k, ko), c in zip(outs[1:], codes[1:]):
            if c == 0:
                assert_same(from_dev(ko, np.uint32), np.sort(k), "good request")
            else:
                assert batched and c == 3


def test_bucket_requests_are_batched(rs, oracle):
    """Small bucket requests with the default bucket count are packed into
    segmented bucket sorts (bs_sort_segmented_*): u32 keys with bounds found
    on the device and u64 keys with values and declared bounds.  With one
    stream, the requests that wait behind the first launch form batches.
    Every result equals the oracle's bucket sort of the request alone."""
    import torch

    reqs = []
    for i in range(40):
        n = 2000 + 1777 * i
        reqs.append((synth.keys_u32(n, i % 7, seed=300 + i), None, {}))
    for i in range(12):
        n = 3000 + 2500 * i
        keys = synth.keys_u64(n, 40, seed=350 + i)
        reqs.append((keys, synth.index_values(n), {"min_key": 0, "max_key": 2**40 - 1}))
    with rs.Server(pool_bytes=2 << 30, num_streams=1, max_batch=16) as srv:
        staged = []
        for keys, vals, bounds in reqs:
            kd = to_dev(keys)
            vd = to_dev(vals) if vals is not None else None
            staged.append((kd, torch.empty_like(kd), vd, torch.empty_like(vd) if vd is not None else None, bounds))
        torch.cuda.synchronize()
        handles = [(srv.submit(kd, ko, vd, vo, algo=rs.RS_ALGO_BUCKET, **b), ko, vo) for kd, ko, vd, vo, b in staged]
        for (t, ko, vo), (keys, vals, bounds) in zip(handles, reqs):
            assert srv.wait(t, 60_000) == 0
            want = oracle.bucket_sort(keys, vals, bounds.get("min_key"), bounds.get("max_key"))
            if vals is None:
                assert_same(from_dev(ko, keys.dtype), want, f"bucket ticket {t}")
            else:
                assert_same(from_dev(ko, keys.dtype), want[0], f"bucket ticket {t} keys")
                assert_same(from_dev(vo, np.uint32), want[1], f"bucket ticket {t} values")
        st = srv.stats()
        assert st.batches >= 2 and st.batched_requests >= 10
