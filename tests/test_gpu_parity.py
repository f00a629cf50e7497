"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars:
  Sobol' integers                      bit-exact
  paths, FP64 path                     rtol 1e-11 (CUDA's normcdfinv and exp
                                       within about 1 ulp, a few ulp per
                                       bridge level)
  paths, mixed (FP32) path             rtol 2e-5: the FP32 uniform (2^-24), the
                                       FP32 quantile (<= 2.4e-6), lg2.approx
                                       (2^-22), the FP32 bridge over <= 10
                                       levels and ex2.approx with exponent
                                       rounding (~6e-7), <~ 1e-5 worst case
  prices (every rule, both precisions) |dP| <= 2e-4 K on identical points
  repeated runs, batch vs single       bit-identical
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from lsm_replay import gpu_fit, gpu_replay, replay_check
from lsm_sensitivity import check_mixed_vs_oracle, fp32_sum_shift

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


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _gpu_paths(amc, ctx, torch, opt, prec):
    ld = amc.amc_path_ld(opt.n_paths)
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.full((opt.n_steps, ld), float("nan"), dtype=dt, device="cuda")
    amc.amc_generate_paths(ctx, opt, prec, S)
    torch.cuda.synchronize()
    return S[:, :opt.n_paths].double().cpu().numpy()


def _gpu_price(amc, ctx, opt, prec):
    return amc.amc_price_american(ctx, opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths,
                                  opt.basis, opt.type, opt.seed, opt.rule, prec)


def _oracle_price(opt):
    return oracle.price(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, basis=opt.basis,
                        type=opt.type, seed=opt.seed, rule=opt.rule)


# ------------------------------------------------------------------ Sobol'
@pytest.mark.parametrize("m,n,seed", [(50, 2 ** 14 + 5, 1), (252, 4099, 2), (365, 1000, 7), (512, 777, 3),
                                      (1, 33, 0)])
def test_sobol_bit_exact(amc, ctx, torch, m, n, seed):
    x = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    amc.amc_sobol(ctx, m, n, seed, x)
    torch.cuda.synchronize()
    got = x.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, oracle.sobol(n, m, seed=seed))


def test_sobol_full_size_sampled_blocks(amc, ctx, torch):
    m, n, seed = 252, 2 ** 20, 2
    x = torch.zeros((m, n), dtype=torch.int32, device="cuda")
    amc.amc_sobol(ctx, m, n, seed, x)
    torch.cuda.synchronize()
    V = oracle.directions(m)
    for i0 in [0, 511, 2 ** 19 - 3, 777777, n - 64]:
        blk = x[:, i0:i0 + 64].cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(blk, oracle.sobol(64, m, i0=i0, seed=seed, V=V))


# ------------------------------------------------------------------ paths
PATH_CASES = [
    workloads.scaled(workloads.single_small(), n_paths=2 ** 14 + 37),
    workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 252, 5000, basis=4, seed=2),
    workloads.Option(90.0, 100.0, 0.03, 0.45, 2.0, 365, 2048, seed=9, type=1),
    workloads.Option(100.0, 95.0, 0.01, 0.1, 0.25, 512, 1000, seed=5),
    workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 100, seed=4),
    workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 2, 33, seed=4),
]


@pytest.mark.parametrize("idx", range(len(PATH_CASES)))
def test_paths_fp64_vs_oracle(amc, ctx, torch, idx):
    opt = PATH_CASES[idx]
    got = _gpu_paths(amc, ctx, torch, opt, amc.AMC_FP64)
    ref = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=0)


@pytest.mark.parametrize("idx", range(len(PATH_CASES)))
def test_paths_mixed_vs_oracle(amc, ctx, torch, idx):
    opt = PATH_CASES[idx]
    got = _gpu_paths(amc, ctx, torch, opt, amc.AMC_MIXED)
    ref = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    rel = np.abs(got / ref - 1.0)
    assert np.isfinite(got).all()
    assert rel.max() < 2e-5, rel.max()


def test_paths_full_size_sampled(amc, ctx, torch):
    opt = workloads.single_large()
    for prec, tol in ((amc.AMC_MIXED, 2e-5), (amc.AMC_FP64, 1e-11)):
        got = _gpu_paths(amc, ctx, torch, opt, prec)
        for first in [0, 123456, opt.n_paths - 300]:
            ref = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, 300, opt.seed, first=first)
            rel = np.abs(got[:, first:first + 300] / ref - 1.0)
            assert rel.max() < tol, (prec, first, rel.max())


# ------------------------------------------------------------------ prices
PRICE_CASES = [
    ("single_small_lsm", workloads.single_small()),
    ("single_small_paper", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, seed=1, rule=1)),
    ("single_small_euro", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, seed=1, rule=2)),
    ("ragged_call_p2", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11)),
    ("ragged_put_p4", workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 100, 30001, basis=4, seed=12)),
    ("one_date", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=13)),
    ("one_date_paper", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=13, rule=1)),
    ("two_dates_p1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 2, 1000, basis=1, seed=14)),
    ("many_dates", workloads.Option(100.0, 110.0, 0.02, 0.4, 2.0, 365, 8192, basis=3, seed=15)),
    ("max_dates", workloads.Option(100.0, 90.0, 0.05, 0.2, 1.0, 512, 3000, basis=3, seed=16)),
    ("tiny_paths", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 5, basis=3, seed=17)),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18)),
    ("big_group", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 60, 2 ** 19 + 3, basis=4, seed=19)),
    ("tiny_vol", workloads.Option(100.0, 100.0, 0.05, 0.01, 1.0, 50, 8192, basis=3, seed=20)),
    ("huge_vol", workloads.Option(100.0, 100.0, 0.05, 1.5, 1.0, 50, 8192, basis=4, seed=21)),
    ("zero_rate", workloads.Option(100.0, 105.0, 0.0, 0.3, 1.0, 50, 8192, basis=3, seed=22)),
    ("negative_rate", workloads.Option(100.0, 95.0, -0.01, 0.25, 2.0, 40, 8192, basis=3, type=1, seed=23)),
    ("short_maturity", workloads.Option(100.0, 100.0, 0.05, 0.3, 0.01, 10, 8192, basis=3, seed=24)),
    ("deep_itm_put", workloads.Option(20.0, 40.0, 0.06, 0.2, 1.0, 50, 8192, basis=3, seed=25)),
    ("long_call", workloads.Option(50.0, 60.0, 0.08, 0.4, 10.0, 120, 8192, basis=4, type=1, seed=26)),
]


# LSM with a cubic over a very wide moneyness range is unstable at FP32
# precision: the oracle's own price moves by more than 2e-4 K under path noise
# at the FP32 paths' error level, and (volatility 150 %) under FP32 sums on
# identical paths (tests/test_fp32_sensitivity.py).  On these two cases the
# mixed sweep on the GPU's own paths is held to the replay check
# (tests/lsm_replay.py: every date's normal equations and the price within the
# FP32 bounds of the kernel's own arithmetic on its own paths).  The free-
# running mixed price of every LSM case goes through check_mixed_vs_oracle:
# within 2e-4 K of the oracle, or, only on an option whose oracle price itself
# moves by more than half that under FP32-level perturbations, the replay check
# and the FP64 price within 2e-4 K.  Besides these two, 512 dates on 3000
# paths is such an option (its oracle price moves 2.0e-4 K under 2e-5 path
# noise, test_many_dates_on_few_paths_are_sensitive_to_fp32_path_noise), and
# so is the 365-date put on 8192 paths, whose oracle price moves 1.2e-4 K
# under FP32 sums on identical paths alone
# (test_a_365_date_put_on_8192_paths_is_unstable_at_fp32_precision): the
# mixed sweep on identical paths may miss the bar there, by its summation
# order, and is then held to the replay check alone.
UNSTABLE_IN_FP32 = {"huge_vol", "long_call"}


@pytest.mark.parametrize("name,opt", PRICE_CASES, ids=[c[0] for c in PRICE_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_price_vs_oracle(amc, ctx, name, opt, prec):
    ref = _oracle_price(opt)
    got = _gpu_price(amc, ctx, opt, prec)
    assert got["status"] == 0
    if prec == 1 and opt.rule == 0:
        check_mixed_vs_oracle(opt, got["price"], ref["price"], lambda: _gpu_price(amc, ctx, opt, 0)["price"],
                              lambda: gpu_replay(amc, ctx, opt))
    else:
        assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (got, ref)
    assert got["degenerate_dates"] == ref["degenerate_dates"]
    assert abs(got["std_err"] - ref["std_err"]) <= 1e-3 * max(ref["std_err"], 1e-12) + 2e-4 * opt.K


@pytest.mark.parametrize("name,opt", PRICE_CASES, ids=[c[0] for c in PRICE_CASES])
def test_mixed_sweep_on_identical_paths(amc, ctx, torch, name, opt):
    """The mixed sweep alone, on the GPU's own FP32 paths.  LSM: the replay
    check (tests/lsm_replay.py) holds every date's regression and the price
    to the FP32 bounds of the kernel's arithmetic given its own decisions;
    on the options where the estimator is stable at FP32 precision the
    price is also within 2e-4 K of the oracle's free-running FP64 sweep on
    the same paths.  The other rules: the oracle on the same paths."""
    Sh, coef, got = gpu_fit(amc, ctx, torch, opt) if opt.rule == 0 else (None, None, None)
    if opt.rule == 0:
        d = replay_check(Sh, opt, coef, got)
        assert d["residual_ratio"] <= 1.0
        ref = oracle.lsm(Sh, opt.type, opt.K, opt.r, opt.T, opt.basis)
        if name not in UNSTABLE_IN_FP32 and abs(got["price"] - ref["price"]) > 2e-4 * opt.K:
            # a miss is allowed only where FP32 sums alone, on identical
            # paths, move the oracle's own price by more than half the bar
            assert fp32_sum_shift(opt) > 1e-4, (got, ref)
        assert got["degenerate_dates"] == ref["degenerate_dates"]
        return
    ld = amc.amc_path_ld(opt.n_paths)
    S = torch.empty((opt.n_steps, ld), dtype=torch.float32, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_generate_paths(ctx, opt, amc.AMC_MIXED, S)
    amc.amc_sweep(ctx, opt, amc.AMC_MIXED, S, res)
    torch.cuda.synchronize()
    got = amc.res_to_dict(res.cpu().numpy())
    Sh = S[:, :opt.n_paths].double().cpu().numpy()
    if opt.rule == 1:
        ref = oracle.paper_ub(Sh, opt.type, opt.S0, opt.K, opt.r, opt.sigma, opt.T)
    else:
        ref = oracle.european(Sh, opt.type, opt.K, opt.r, opt.T)
    assert got["status"] == 0
    assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (got, ref)
    assert got["degenerate_dates"] == ref["degenerate_dates"]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_price_full_size_vs_oracle(amc, ctx, prec):
    opt = workloads.single_large()
    ref = _oracle_price(opt)
    got = _gpu_price(amc, ctx, opt, prec)
    assert got["status"] == 0
    assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (got, ref)


# ------------------------------------------------------------------ invariants
def test_run_to_run_bit_identical(amc, ctx):
    for opt in (workloads.single_small(), workloads.scaled(workloads.single_large(), n_paths=2 ** 18)):
        a = _gpu_price(amc, ctx, opt, amc.AMC_MIXED)
        b = _gpu_price(amc, ctx, opt, amc.AMC_MIXED)
        assert a["price"] == b["price"] and a["std_err"] == b["std_err"]


def test_batch_equals_single(amc, ctx):
    opts = [c[1] for c in PRICE_CASES if c[1].n_paths <= 2 ** 16] + workloads.batch_options(n=6)
    opts = [workloads.scaled(o, n_paths=min(o.n_paths, 2 ** 15)) for o in opts]
    for prec in (amc.AMC_MIXED, amc.AMC_FP64):
        batch = amc.amc_price_batch(ctx, opts, prec)
        for o, b in zip(opts, batch):
            s = _gpu_price(amc, ctx, o, prec)
            assert b["price"] == s["price"] and b["std_err"] == s["std_err"], (o, b, s)


def test_full_batch_sampled_vs_oracle_and_alone(amc, ctx):
    """The 4096-option batch at full size (2^14..2^18 paths, 12..365 dates),
    mixed precision: a seeded sample of 16 options equals the option priced
    alone bit for bit, and a seeded 1 % sample is within 2e-4 K of the
    oracle on the same points, with equal degenerate counts.  Options on
    which LSM is unstable at FP32 precision (deep in-the-money calls with a
    wide moneyness range) are held to the oracle's own FP32 sensitivity, and
    their FP64 GPU price to 2e-4 K, while the mixed sweep is held to the
    replay check on its own paths, priced alone, whose result equals the
    batch's bit for bit (check_mixed_vs_oracle)."""
    opts = workloads.batch_options()
    res = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED)
    assert all(r["status"] == 0 for r in res)
    for i in np.random.default_rng(43).choice(len(opts), size=16, replace=False):
        s = _gpu_price(amc, ctx, opts[i], amc.AMC_MIXED)
        assert res[i]["price"] == s["price"] and res[i]["std_err"] == s["std_err"], (i, res[i], s)

    def replay_alone(i):
        s = _gpu_price(amc, ctx, opts[i], amc.AMC_MIXED)
        assert res[i]["price"] == s["price"], (i, res[i], s)
        gpu_replay(amc, ctx, opts[i])

    for i in np.random.default_rng(44).choice(len(opts), size=len(opts) // 100, replace=False):
        o = opts[i]
        ref = _oracle_price(o)
        check_mixed_vs_oracle(o, res[i]["price"], ref["price"], lambda: _gpu_price(amc, ctx, o, amc.AMC_FP64)["price"],
                              lambda: replay_alone(i))
        assert res[i]["degenerate_dates"] == ref["degenerate_dates"]


def test_batch_option_659_replay(amc, ctx):
    """Batch option 659, a deep in-the-money call with a wide moneyness range
    on which LSM is unstable at FP32 precision: the replay check on its own
    paths, and the batch result equal to the option priced alone."""
    o = workloads.batch_options()[659]
    d = gpu_replay(amc, ctx, o)
    assert d["residual_ratio"] <= 1.0 and d["price_ratio"] <= 1.0
    b = amc.amc_price_batch(ctx, [o], amc.AMC_MIXED)[0]
    assert b["price"] == _gpu_price(amc, ctx, o, amc.AMC_MIXED)["price"]


def test_full_greeks_sampled_vs_oracle(amc, ctx):
    """The 1024-put Greeks workload at full size (2^18 paths, 100 dates),
    mixed precision: a seeded 1 % sample against the oracle's frozen-boundary
    pathwise price, delta and vega on the same points (bars as above)."""
    opts = workloads.greeks_options()
    p, d, v = amc.amc_greeks(ctx, opts, amc.AMC_MIXED)
    for i in np.random.default_rng(45).choice(len(opts), size=len(opts) // 100, replace=False):
        o = opts[i]
        g = oracle.greeks(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                          seed=o.seed, rule=o.rule)
        if abs(p[i] - g["price"]) > 2e-4 * o.K:      # unstable at FP32 precision: FP64 Greeks carry the bars
            check_mixed_vs_oracle(o, p[i], g["price"], lambda: amc.amc_greeks(ctx, [o], amc.AMC_FP64)[0][0],
                                  lambda: gpu_replay(amc, ctx, o))
            _, dd, vv = amc.amc_greeks(ctx, [o], amc.AMC_FP64)
            assert abs(dd[0] - g["delta"]) <= 1e-9 + 5e-4 and abs(vv[0] - g["vega"]) <= 0.1, (i, dd, vv, g)
            continue
        assert abs(d[i] - g["delta"]) <= 2e-3 + 5e-4, (i, d[i], g)
        assert abs(v[i] - g["vega"]) <= 0.2 + 5e-2 * max(1.0, abs(g["vega"])), (i, v[i], g)


def test_device_entry_points_match_host_call(amc, ctx, torch):
    opt = workloads.single_small()
    for prec in (amc.AMC_MIXED, amc.AMC_FP64):
        ld = amc.amc_path_ld(opt.n_paths)
        S = torch.empty((opt.n_steps, ld), dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        amc.amc_price_device(ctx, opt, prec, S, res)
        torch.cuda.synchronize()
        dev = amc.res_to_dict(res.cpu().numpy())
        host = _gpu_price(amc, ctx, opt, prec)
        assert dev["price"] == host["price"]


# ------------------------------------------------------------------ Greeks
def test_greeks_vs_oracle_pathwise(amc, ctx):
    opts = [workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 2 ** 14, basis=3, seed=5),
            workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 25, 2 ** 13, basis=4, seed=6, rule=2),
            workloads.Option(110.0, 100.0, 0.02, 0.25, 0.5, 12, 5000, basis=3, type=1, seed=7)]
    for prec, tol in ((amc.AMC_FP64, 1e-9), (amc.AMC_MIXED, 2e-3)):
        p, d, v = amc.amc_greeks(ctx, opts, prec)
        for k, o in enumerate(opts):
            g = oracle.greeks(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                              seed=o.seed, rule=o.rule)
            assert abs(p[k] - g["price"]) <= 2e-4 * o.K
            assert abs(d[k] - g["delta"]) <= tol + 5e-4, (prec, k, d[k], g["delta"])
            assert abs(v[k] - g["vega"]) <= tol * 100 + 5e-2 * max(1.0, abs(g["vega"])) * (prec == 1) + 1e-6, \
                (prec, k, v[k], g["vega"])


def test_greeks_vs_central_differences(amc, ctx):
    o = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 2 ** 16, basis=3, seed=5)
    p, d, v = amc.amc_greeks(ctx, [o], amc.AMC_FP64)
    bS, bv = 1e-3 * o.S0, 1e-3 * o.sigma
    f = lambda **kw: _gpu_price(amc, ctx, workloads.Option(**{**o.as_dict(), **kw}), amc.AMC_FP64)["price"]
    fd_d = (f(S0=o.S0 + bS) - f(S0=o.S0 - bS)) / (2 * bS)
    fd_v = (f(sigma=o.sigma + bv) - f(sigma=o.sigma - bv)) / (2 * bv)
    assert abs(d[0] - fd_d) < 0.02 * abs(fd_d) + 5e-3
    assert abs(v[0] - fd_v) < 0.05 * abs(fd_v) + 0.2


def test_autograd_gradients_are_the_adjoint_greeks(amc, ctx):
    """american_price through torch.autograd: the price and the gradients in
    S0 and sigma are the adjoint kernel's price, delta and vega bit for bit,
    and the gradient agrees with central differences of GPU prices."""
    import torch

    from paper_1205_0106_gb300.autograd import american_price
    opts = [workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 2 ** 16, basis=3, seed=5),
            workloads.Option(44.0, 40.0, 0.06, 0.4, 2.0, 25, 2 ** 15, basis=3, seed=6)]
    for prec in (amc.AMC_FP64, amc.AMC_MIXED):
        S0 = torch.tensor([o.S0 for o in opts], dtype=torch.float64, device="cuda", requires_grad=True)
        sig = torch.tensor([o.sigma for o in opts], dtype=torch.float64, device="cuda", requires_grad=True)
        p = american_price(ctx, S0, sig, K=40.0, r=0.06, T=[o.T for o in opts], n_steps=[o.n_steps for o in opts],
                           n_paths=[o.n_paths for o in opts], basis=3, seed=[o.seed for o in opts], prec=prec)
        assert p.device == S0.device
        p.sum().backward()
        ref_p, ref_d, ref_v = amc.amc_greeks(ctx, opts, prec)
        assert np.array_equal(p.detach().cpu().numpy(), ref_p)
        assert np.array_equal(S0.grad.cpu().numpy(), ref_d) and np.array_equal(sig.grad.cpu().numpy(), ref_v)
    o = opts[0]
    bS = 1e-3 * o.S0
    f = lambda s: _gpu_price(amc, ctx, workloads.Option(**{**o.as_dict(), "S0": s}), amc.AMC_FP64)["price"]
    fd = (f(o.S0 + bS) - f(o.S0 - bS)) / (2 * bS)
    S0 = torch.tensor([o.S0], dtype=torch.float64, requires_grad=True)
    american_price(ctx, S0, o.sigma, o.K, o.r, o.T, o.n_steps, o.n_paths, seed=o.seed, prec=amc.AMC_FP64).backward()
    assert abs(S0.grad.item() - fd) < 0.02 * abs(fd) + 5e-3


# ------------------------------------------------------------------ failures
def test_device_wait_timeout_is_reported_and_context_survives(amc, ctx):
    opt = workloads.scaled(workloads.single_large(), n_paths=2 ** 18, n_steps=20)
    ctx.set_timeout(0.02)
    try:
        ctx.inject(1, 7)
        with pytest.raises(amc.AmcError) as ei:
            _gpu_price(amc, ctx, opt, amc.AMC_MIXED)
        assert ei.value.code == amc.AMC_ETIMEOUT
    finally:
        ctx.set_timeout(2.0)
    ok = _gpu_price(amc, ctx, workloads.single_small(), amc.AMC_MIXED)
    assert ok["status"] == 0 and abs(ok["price"] - 4.46) < 0.05


def test_allocation_failure_is_reported(amc, ctx):
    ctx.inject(2)
    with pytest.raises(amc.AmcError) as ei:
        _gpu_price(amc, ctx, workloads.single_small(), amc.AMC_MIXED)
    assert ei.value.code == amc.AMC_ENOMEM
    assert _gpu_price(amc, ctx, workloads.single_small(), amc.AMC_MIXED)["status"] == 0


def test_invalid_arguments_rejected_before_device_work(amc, ctx):
    bad = workloads.scaled(workloads.single_small(), n_steps=0)
    with pytest.raises(amc.AmcError) as ei:
        _gpu_price(amc, ctx, bad, amc.AMC_MIXED)
    assert ei.value.code == amc.AMC_EINVAL
    with pytest.raises(amc.AmcError):
        amc.amc_greeks(ctx, [workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 5, 100, rule=1)], amc.AMC_MIXED)
