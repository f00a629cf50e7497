"""Stale cross-CTA exchange data on the batch and serving paths.

The mixed-precision LSM sweep of an option above 2^18 paths sums each date's
per-CTA partials through 64-bit exchange units in global memory: an FP32
payload under a 32-bit tag made of the launch's tag and the exchange index,
polled until every tag matches (smaller options exchange on chip, within
one thread-block cluster, and the Greeks variant always uses the units).  The
batch and serving launches take their units from the context arena, whose
bytes held earlier requests' paths, partial sums and units.  The library
clears a launch's units before the launch; these tests make the worst case
happen on purpose: the next launch reuses the tag of an earlier launch with
the same layout (amc_ctx_inject kind 4), so every unit that launch left
behind carries exactly the tag the new launch waits for, but other values.
The results must still equal the options priced alone, bit for bit, and the
oracle on the same points.  Only wrong data could come of a failure here,
never a fault or a hang: every unit address is inside the launch's own
arena allocation and every wait is bounded.
"""
import time

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

REPLAYED_TAG = 0x3FF00          # any tag in 1 .. 2^22 - 1; this one is the high word of doubles near 1.0 >> 10


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


def _layout(n, seed, n_paths, max_steps=60):
    """n mixed-LSM options (dates up to max_steps, type and basis from the
    batch draw, n_paths paths each) and a second set with the same layouts
    but other prices, rates and shifts (moneyness 0.9..1.1, volatility
    15..35 %, where the estimator is stable at FP32 precision).  Above 2^18
    paths the mixed sweep exchanges through tagged units in the arena (at
    most 2^18, one cluster per option exchanges on chip)."""
    base = workloads.batch_options(n=n)
    rng = np.random.default_rng(seed)
    a, b = [], []
    for k, o in enumerate(base):
        o = workloads.scaled(o, n_paths=n_paths, n_steps=min(o.n_steps, max_steps))
        a.append(o)
        K = float(rng.uniform(80, 120))
        b.append(workloads.Option(K * float(rng.uniform(0.9, 1.1)), K, float(rng.uniform(0, 0.08)),
                                  float(rng.uniform(0.15, 0.35)), float(rng.uniform(0.25, 2.0)), o.n_steps, o.n_paths,
                                  basis=o.basis, type=o.type, seed=o.seed + 7919, rule=o.rule))
    return a, b


def _alone(amc, ctx, o, prec=1):
    return amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                  o.rule, prec)


def test_batch_with_replayed_tags_equals_alone_and_oracle(amc):
    first, second = _layout(24, 101, 300000)
    with amc.Context(0, arena_bytes=4 << 30) as ctx:
        alone = [_alone(amc, ctx, o) for o in second]
        ctx.inject(4, REPLAYED_TAG)
        res_first = amc.amc_price_batch(ctx, first, amc.AMC_MIXED)
        ctx.inject(4, REPLAYED_TAG)          # same tags, same waves, same arena bytes
        res = amc.amc_price_batch(ctx, second, amc.AMC_MIXED)
    assert all(r["status"] == 0 for r in res_first + res)
    for o, r, s in zip(second, res, alone):
        assert r["price"] == s["price"] and r["std_err"] == s["std_err"], (o, r, s)
    for k in (0, 5, 11, 23):
        o = second[k]
        ref = oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                           seed=o.seed)
        assert abs(res[k]["price"] - ref["price"]) <= 2e-4 * o.K, (k, o, res[k], ref)
        assert res[k]["degenerate_dates"] == ref["degenerate_dates"]


def test_greeks_with_replayed_tags_equal_alone(amc):
    first, second = _layout(8, 102, 2 ** 15, max_steps=365)
    first = [workloads.Option(**{**o.as_dict(), "type": workloads.PUT}) for o in first]
    second = [workloads.Option(**{**o.as_dict(), "type": workloads.PUT}) for o in second]
    with amc.Context(0, arena_bytes=1 << 30) as ctx:
        p0, d0, v0 = amc.amc_greeks(ctx, second, amc.AMC_MIXED)
        ctx.inject(4, REPLAYED_TAG)
        amc.amc_greeks(ctx, first, amc.AMC_MIXED)
        ctx.inject(4, REPLAYED_TAG)
        p, d, v = amc.amc_greeks(ctx, second, amc.AMC_MIXED)
    assert np.array_equal(p, p0) and np.array_equal(d, d0) and np.array_equal(v, v0)


def test_served_mix_with_replayed_tags_equals_alone(amc):
    """A served mix whose first launch reuses the tag of a batch launch that
    ran just before it on the same arena: every result equals alone."""
    first, second = _layout(16, 103, 300000)
    with amc.Context(0, arena_bytes=4 << 30) as ctx:
        alone = [_alone(amc, ctx, o) for o in second]
        ctx.inject(4, REPLAYED_TAG)
        amc.amc_price_batch(ctx, first, amc.AMC_MIXED)
        ctx.inject(4, REPLAYED_TAG)
        amc.amc_serve_start(ctx, slots=2, max_batch=4, prec=amc.AMC_MIXED)
        tickets = {}
        for i, o in enumerate(second):
            tickets[amc.amc_serve_submit(ctx, o)] = i
            time.sleep(0.0003)
        got = {}
        deadline = time.time() + 120
        while len(got) < len(second) and time.time() < deadline:
            for t, r, _ in amc.amc_serve_drain(ctx):
                got[tickets[t]] = r
            time.sleep(0.002)
        amc.amc_serve_stop(ctx)
    assert len(got) == len(second)
    for i, r in got.items():
        assert r["status"] == 0
        assert r["price"] == alone[i]["price"] and r["std_err"] == alone[i]["std_err"], (i, r, alone[i])


def test_replayed_tag_is_validated(amc):
    with amc.Context(0, arena_bytes=64 << 20) as ctx:
        for bad in (0, 1 << 22, -3):
            with pytest.raises(amc.AmcError) as ei:
                ctx.inject(4, bad)
            assert ei.value.code == amc.AMC_EINVAL
        ctx.inject(0)
