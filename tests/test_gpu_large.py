"""Options larger than the register-resident sweeps hold (about 1.2 M paths
on 152 SMs): the streaming LSM sweep (cash flows in device memory, one pass
and one solve per date) and the pathwise rules on an uncapped grid, against
the FP64 oracle on identical points, through the C ABI.

Bars: |dP| <= 2e-4 K (mixed) and 1e-10 K (FP64) with equal degenerate-date
counts; the streaming sweep forced on small options (context injection
kind 3) over the edge cases of the LSM parity suite, in FP64 within 1e-10 K
of the oracle and of the register-resident sweep on the same paths, in
mixed precision each sweep against the oracle (where the estimator is
unstable at FP32 precision, each sweep held to the replay check on its own
paths instead, check_mixed_vs_oracle);
Greeks beyond the register-resident sizes are refused.
"""
import pytest

import oracle
import workloads
from lsm_replay import gpu_replay
from lsm_sensitivity import check_mixed_vs_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


@pytest.fixture(scope="module")
def ctx(amc):
    c = amc.Context(0, arena_bytes=12 << 30)
    yield c
    c.close()


def _gpu(amc, ctx, o, prec):
    return amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                  o.rule, prec)


def _oracle(o):
    return oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type, seed=o.seed,
                        rule=o.rule)


LARGE = [
    ("lsm_put_2p21", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21, basis=4, seed=51)),
    ("lsm_call_ragged", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 30, 2 ** 21 + 12345, basis=3, type=1,
                                         seed=52)),
    ("paper_rule_2p21", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21, seed=53,
                                         rule=workloads.RULE_PAPER_UB)),
    ("european_2p21", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21 + 7, seed=54,
                                       rule=workloads.RULE_EUROPEAN)),
]


@pytest.mark.parametrize("name,opt", LARGE, ids=[c[0] for c in LARGE])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_large_option_vs_oracle(amc, ctx, name, opt, prec):
    got = _gpu(amc, ctx, opt, prec)
    ref = _oracle(opt)
    tol = 1e-10 if prec == amc.AMC_FP64 else 2e-4
    assert got["status"] == 0
    assert abs(got["price"] - ref["price"]) <= tol * opt.K, (got, ref)
    assert abs(got["std_err"] - ref["std_err"]) <= 1e-3 * ref["std_err"] + tol * opt.K
    if opt.rule == workloads.RULE_LSM:
        assert got["degenerate_dates"] == ref["degenerate_dates"]


def test_four_million_paths(amc, ctx):
    """A 2^22-path, 100-date put (1.7 GB of FP32 paths), mixed precision."""
    opt = workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 100, 2 ** 22, basis=4, seed=55)
    got = _gpu(amc, ctx, opt, amc.AMC_MIXED)
    ref = _oracle(opt)
    assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (got, ref)


FORCED = [
    ("ls_table1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=1)),
    ("ragged_call_p2", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11)),
    ("put_p4_m100", workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 100, 30001, basis=4, seed=12)),
    ("basis_1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 5000, basis=1, seed=14)),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18)),
    ("one_date", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=13)),
    ("two_dates", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 2, 999, seed=13)),
    ("five_paths", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 5, 5, basis=2, seed=16)),
    ("max_dates", workloads.Option(100.0, 110.0, 0.02, 0.4, 2.0, 512, 3000, basis=3, seed=17)),
]


@pytest.mark.parametrize("name,opt", FORCED, ids=[c[0] for c in FORCED])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_streaming_sweep_forced_on_small_options(amc, ctx, name, opt, prec):
    ctx.inject(3)
    got = _gpu(amc, ctx, opt, prec)
    ref = _oracle(opt)
    alone = _gpu(amc, ctx, opt, prec)                    # the register-resident sweep, same points
    assert got["status"] == 0
    assert got["degenerate_dates"] == ref["degenerate_dates"]
    if prec == amc.AMC_FP64:
        assert abs(got["price"] - ref["price"]) <= 1e-10 * opt.K, (got, ref)
        assert abs(got["price"] - alone["price"]) <= 1e-10 * opt.K, (got, alone)
    else:
        # each mixed sweep against the oracle; an FP32-sensitive option (the 512-date case: few
        # in-the-money paths per regression) is held to the oracle's own FP32 sensitivity
        fp64 = lambda: _gpu(amc, ctx, opt, amc.AMC_FP64)["price"]
        check_mixed_vs_oracle(opt, got["price"], ref["price"], fp64, lambda: gpu_replay(amc, ctx, opt, streaming=True))
        check_mixed_vs_oracle(opt, alone["price"], ref["price"], fp64, lambda: gpu_replay(amc, ctx, opt))


def test_streaming_sweep_is_deterministic_and_writes_the_boundary(amc, ctx):
    import torch
    opt = workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21, basis=4, seed=51)
    a = _gpu(amc, ctx, opt, amc.AMC_MIXED)
    b = _gpu(amc, ctx, opt, amc.AMC_MIXED)
    assert a["price"] == b["price"] and a["std_err"] == b["std_err"]
    # fitted boundary of a large option: the same flags as the oracle's fit, and a value on
    # independent points within the price bar of the oracle's
    fit, val = amc.amc_price_oos(ctx, opt, 77, amc.AMC_MIXED)
    rfit, rval = oracle.price_oos(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, basis=opt.basis,
                                  type=opt.type, seed=opt.seed, value_seed=77)
    assert abs(fit["price"] - rfit["price"]) <= 2e-4 * opt.K
    assert abs(val["price"] - rval["price"]) <= 2e-4 * opt.K, (val, rval)
    assert val["degenerate_dates"] == rval["degenerate_dates"]
    del torch


def test_large_greeks_are_refused(amc, ctx):
    opt = workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 50, 2 ** 21, basis=4, seed=51)
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_greeks(ctx, [opt], amc.AMC_MIXED)
    assert ei.value.code == amc.AMC_EINVAL
