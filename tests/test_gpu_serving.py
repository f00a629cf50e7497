"""Serving loop on the GPU: continuous batching, admission by memory, and
the same result for a request whether it is served alone or in a mix."""
import threading
import time

import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


def _mix(n):
    opts = workloads.serving_requests(rate=2000.0, duration=1.0, seed=4)[1][:n]
    # keep the test quick: at most 2^15 paths, all dates as drawn
    return [workloads.scaled(o, n_paths=min(o.n_paths, 2 ** 15)) for o in opts]


def _alone(amc, ctx, o, prec):
    return amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                  o.rule, prec)


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "fp64"])
def test_served_results_equal_alone(amc, prec):
    opts = _mix(40 if prec == 1 else 12)
    with amc.Context(0, arena_bytes=3 << 30) as ctx:
        alone = [_alone(amc, ctx, o, prec) for o in opts]
        amc.amc_serve_start(ctx, slots=3, max_batch=16, prec=prec)
        tickets = {}
        lock = threading.Lock()

        def submit(part):
            for i in part:
                t = amc.amc_serve_submit(ctx, opts[i])
                with lock:
                    tickets[t] = i
                time.sleep(0.0005)

        ths = [threading.Thread(target=submit, args=(range(k, len(opts), 2),)) for k in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        got = {}
        deadline = time.time() + 120
        while len(got) < len(opts) and time.time() < deadline:
            for t, r, lat in amc.amc_serve_drain(ctx):
                got[tickets[t]] = (r, lat)
            time.sleep(0.002)
        stats = amc.amc_serve_stats_get(ctx)
        amc.amc_serve_stop(ctx)
    assert len(got) == len(opts)
    assert stats["completed"] == len(opts) and stats["batches"] >= 2
    for i, (r, lat) in got.items():
        assert r["status"] == 0 and lat > 0
        assert r["price"] == alone[i]["price"] and r["std_err"] == alone[i]["std_err"], (i, r, alone[i])


def test_admission_by_memory_and_busy_context(amc):
    with amc.Context(0, arena_bytes=256 << 20) as ctx:
        amc.amc_serve_start(ctx, slots=2, max_batch=8)
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_serve_submit(ctx, workloads.single_large())          # 1.06 GB of paths > 128 MB slot
        assert ei.value.code == amc.AMC_EBUSY
        o = workloads.single_small()
        with pytest.raises(amc.AmcError) as ei:
            _alone(amc, ctx, o, amc.AMC_MIXED)                           # context owned by the server
        assert ei.value.code == amc.AMC_EBUSY
        t = amc.amc_serve_submit(ctx, o)
        for _ in range(10000):
            res = amc.amc_serve_poll(ctx, t)
            if res is not None:
                break
            time.sleep(0.001)
        amc.amc_serve_stop(ctx)
        assert res is not None and res[0]["status"] == 0 and abs(res[0]["price"] - 4.46) < 0.05
        # after stop the context prices directly again
        assert _alone(amc, ctx, o, amc.AMC_MIXED)["price"] == res[0]["price"]
