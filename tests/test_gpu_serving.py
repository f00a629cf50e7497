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


def test_served_stream_vs_alone_fp64_and_oracle(amc):
    """A full-size 1-second Poisson stream of the serving workload (about
    2000 requests, 2^14..2^18 paths, 12..365 dates), served in mixed
    precision: every served result equals the request priced alone, bit for
    bit; a seeded 5 % sample is within 2e-4 K of the all-FP64 GPU path and a
    seeded 1 % sample within 2e-4 K of the FP64 oracle on the same points,
    except where LSM is unstable at FP32 precision on the request, whose
    mixed sweep is then held to the replay check on its own paths and its
    FP64 GPU price to 2e-4 K (check_mixed_vs_oracle)."""
    import numpy as np

    import oracle
    from lsm_replay import gpu_replay
    from lsm_sensitivity import check_mixed_vs_oracle
    _, opts = workloads.serving_requests(rate=2000.0, duration=1.0, seed=4)
    with amc.Context(0, arena_bytes=24 << 30) as ctx:
        amc.amc_serve_start(ctx, slots=3, max_batch=128, prec=amc.AMC_MIXED)
        tickets = {amc.amc_serve_submit(ctx, o): i for i, o in enumerate(opts)}
        got = {}
        deadline = time.time() + 300
        while len(got) < len(opts) and time.time() < deadline:
            for t, r, lat in amc.amc_serve_drain(ctx):
                got[tickets[t]] = r
            time.sleep(0.002)
        amc.amc_serve_stop(ctx)
        assert len(got) == len(opts)
        for i, o in enumerate(opts):
            a = _alone(amc, ctx, o, amc.AMC_MIXED)
            assert got[i]["status"] == 0
            assert got[i]["price"] == a["price"] and got[i]["std_err"] == a["std_err"], (i, got[i], a)
        fp64 = {}
        for i in np.random.default_rng(41).choice(len(opts), size=len(opts) // 20, replace=False):
            fp64[i] = _alone(amc, ctx, opts[i], amc.AMC_FP64)["price"]
        sample = np.random.default_rng(42).choice(len(opts), size=len(opts) // 100, replace=False)
        for i in sample:
            if i not in fp64:
                fp64[i] = _alone(amc, ctx, opts[i], amc.AMC_FP64)["price"]
    for i, f in fp64.items():
        o = opts[i]
        if abs(got[i]["price"] - f) > 2e-4 * o.K:    # only where LSM is unstable at FP32 precision
            ref = oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                               seed=o.seed, rule=o.rule)
            with amc.Context(0, arena_bytes=2 << 30) as c2:
                check_mixed_vs_oracle(o, got[i]["price"], ref["price"], lambda: f, lambda: gpu_replay(amc, c2, o))
    for i in sample:
        o = opts[i]
        ref = oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                           seed=o.seed, rule=o.rule)
        with amc.Context(0, arena_bytes=2 << 30) as c2:
            check_mixed_vs_oracle(o, got[i]["price"], ref["price"], lambda: fp64[i], lambda: gpu_replay(amc, c2, o))
        assert got[i]["degenerate_dates"] == ref["degenerate_dates"]


def test_cancel_a_queued_request(amc):
    """One slot busy with a large request: a request queued behind it can be
    cancelled (it finishes at once with AMC_ECANCELED and never runs); the
    running one cannot (AMC_EBUSY) and completes with its normal result;
    an unknown ticket gives AMC_ENOTFOUND; the other queued requests still
    run and equal their results alone."""
    big = workloads.single_large()
    small = [workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=40 + k) for k in range(3)]
    with amc.Context(0, arena_bytes=4 << 30) as ctx:
        alone = [_alone(amc, ctx, o, amc.AMC_MIXED) for o in small + [big]]
        amc.amc_serve_start(ctx, slots=1, max_batch=8, prec=amc.AMC_MIXED)
        t_big = amc.amc_serve_submit(ctx, big)
        deadline = time.time() + 30
        while amc.amc_serve_stats_get(ctx)["launched"] < 1 and time.time() < deadline:
            time.sleep(0.0002)
        tickets = [amc.amc_serve_submit(ctx, o) for o in small]
        amc.amc_serve_cancel(ctx, tickets[1])
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_serve_cancel(ctx, t_big)
        assert ei.value.code == amc.AMC_EBUSY
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_serve_cancel(ctx, 987654321)
        assert ei.value.code == amc.AMC_ENOTFOUND
        got = {}
        while len(got) < 4 and time.time() < deadline:
            for t, r, lat in amc.amc_serve_drain(ctx):
                got[t] = r
            time.sleep(0.002)
        stats = amc.amc_serve_stats_get(ctx)
        amc.amc_serve_stop(ctx)
    assert got[tickets[1]]["status"] == amc.AMC_ECANCELED
    assert stats["cancelled"] == 1 and stats["launched"] == 3
    for k in (0, 2):
        assert got[tickets[k]]["status"] == 0 and got[tickets[k]]["price"] == alone[k]["price"]
    assert got[t_big]["status"] == 0 and got[t_big]["price"] == alone[3]["price"]
