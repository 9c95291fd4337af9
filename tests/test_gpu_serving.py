"""The continuous-batching server (rs_server_*): every request's result is
the same alone and in a mix of concurrently running requests (exact
equality), requests admitted while others run overlap on the GPU, the memory
budget bounds admission, and oversized or malformed requests fail cleanly."""
import random
import threading
import time

import numpy as np
import pytest

from oracle import exact
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import assert_full_size, rand_bipoly

pytestmark = pytest.mark.gpu


def mixed_requests(seed, n, deg_lo=3, deg_hi=12, bits_lo=16, bits_hi=128):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        df, dg = int(rng.integers(deg_lo, deg_hi + 1)), int(rng.integers(deg_lo, deg_hi + 1))
        b = int(rng.integers(bits_lo, bits_hi + 1))
        L = -(-b // 32)
        out.append((inputs.dense_total_degree(rng, df, b, L), inputs.dense_total_degree(rng, dg, b, L)))
    return out


def test_results_same_alone_and_in_the_mix():
    reqs = mixed_requests(40, 48)
    big = inputs.workload_single(1)[0]  # keeps the GPU busy while the others arrive
    with rs.Context(device=0) as alone_ctx:
        alone = [alone_ctx.resultant_y(f, g) for f, g in reqs]
    with rs.Context(device=0) as ctx:
        srv = rs.Server(ctx, max_inflight=4, max_batch=8)
        tickets = {}
        tb = srv.submit(*big)

        def producer(lo, hi):
            for i in range(lo, hi):
                tickets[i] = srv.submit(*reqs[i])
                time.sleep(0.0005)
        th = [threading.Thread(target=producer, args=(k, k + 12)) for k in range(0, 48, 12)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = {}
        lat = []
        for i, t in tickets.items():
            R, ms = srv.wait(t)
            got[i] = R
            lat.append(ms)
        Rbig, _ = srv.wait(tb)
        st = srv.stats()
        srv.stop()
    for i, (f, g) in enumerate(reqs):
        assert got[i] == alone[i], f"request {i} differs between alone and mixed runs"
    from oracle import modular
    assert [got[i] for i in range(48)] == modular.resultants(reqs)  # every request against O2
    for i in range(0, 48, 8):  # and a sample against the exact oracle O1
        f, g = reqs[i]
        assert got[i] == exact.resultant_y(f.to_ints(), g.to_ints())
    assert_full_size("c1_single", [Rbig], [big])
    assert st["completed"] == 49 and st["failed"] == 0
    assert st["peak_inflight_batches"] >= 2  # micro-batches overlapped on the device
    assert st["batches"] >= 2 and all(x > 0 for x in lat)


def test_memory_budget_bounds_admission():
    reqs = mixed_requests(41, 12, deg_lo=6, deg_hi=10)
    with rs.Context(device=0) as ctx:
        alone = [ctx.resultant_y(f, g) for f, g in reqs]
        srv = rs.Server(ctx, max_inflight=3, max_batch=64, mem_limit_bytes=600_000)
        ts = [srv.submit(f, g) for f, g in reqs]
        seen_max = 0
        done = {}
        while len(done) < len(ts):
            st = srv.stats()
            seen_max = max(seen_max, st["mem_used"])
            assert st["mem_used"] <= st["mem_limit"]
            for i, t in enumerate(ts):
                if i not in done:
                    r = srv.poll(t)
                    if r is not None:
                        done[i] = r[0]
        st = srv.stats()
        assert st["batches"] >= 2  # the budget forced several micro-batches
        # a request that can never fit the budget fails, the server keeps going
        huge = inputs.workload_single(1, deg=40)[0]  # about 5 MB of images alone
        t = srv.submit(*huge)
        with pytest.raises(rs.RsError) as e:
            srv.wait(t)
        assert e.value.code == -3
        t2 = srv.submit(*reqs[0])
        assert srv.wait(t2)[0] == alone[0]
        srv.stop()
    assert [done[i] for i in range(len(ts))] == alone


def test_errors_and_timeouts():
    with rs.Context(device=0) as ctx:
        srv = rs.Server(ctx)
        rng = random.Random(5)
        bad = [[rng.randint(1, 9) for _ in range(73)]]  # y-degree 72 > RS_MAX_DEG_Y
        with pytest.raises(rs.RsError) as e:
            srv.submit(bad, [[1, 1]])
        assert e.value.code == -6
        big = inputs.workload_single(1)[0]
        t = srv.submit(*big)
        r = srv.wait(t, timeout_us=0)  # almost surely still running
        if r is None:
            r = srv.wait(t)
        assert r is not None
        srv.stop()


def test_serving_workload_sample_through_the_server():
    """The first 64 requests of the serving stream (total degrees 8..64,
    16..128-bit coefficients) through the server: each equals the batched
    result bit for bit, and every coefficient equals the oracle O2's."""
    pairs, _ = inputs.workload_serving(4, n=64)
    with rs.Context(device=0) as ctx:
        batched = ctx.resultant_batch(pairs)
        srv = rs.Server(ctx, max_inflight=4, max_batch=16)
        tickets = [srv.submit(f, g) for f, g in pairs]
        got = [srv.wait(t, timeout_us=120_000_000)[0] for t in tickets]
        st = srv.stats()
        srv.stop()
    assert st["failed"] == 0 and st["completed"] == 64
    for i, R in enumerate(got):
        assert R == batched[i], f"request {i}: server and batch differ"
    assert_full_size("c4_serving_first512", got, pairs)


def test_request_log(tmp_path):
    """rs_server_set_log: one JSON line per finished request, with ordered
    times and the planner's K and D."""
    import json
    rng = random.Random(61)
    pairs = [(rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bits=30),
              rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bits=30)) for _ in range(20)]
    path = tmp_path / "requests.jsonl"
    with rs.Context(device=0) as c:
        srv = rs.Server(c)
        srv.set_log(str(path))
        tickets = [srv.submit(f, g) for f, g in pairs]
        for t in tickets:
            srv.wait(t)
        srv.stop()
    recs = {r["ticket"]: r for r in map(json.loads, path.read_text().splitlines())}
    assert sorted(recs) == sorted(tickets)
    for t, (f, g) in zip(tickets, pairs):
        r, b = recs[t], rs.result_bound(f, g)
        assert r["status"] == 0 and 0 <= r["submit_us"] <= r["admit_us"] <= r["done_us"]
        assert (r["K"], r["D"]) == (b["primes"], b["deg"]) and r["footprint"] > 0
