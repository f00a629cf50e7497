"""Binary16 moneyness path storage (AMC_MIXED16) through the C ABI.

The path array holds y = S/K - 1 in IEEE binary16 instead of S in FP32
(half the bytes); path generation writes it and the mixed LSM sweeps (the
cluster sweep, the L2-exchange sweep and the streaming sweep of large
options) read it.  Bars:
  paths        within one binary16 unit in the last place of the FP32
               path's moneyness plus the FP32 roundings of the two paths'
               exponents, and within a binary16 unit plus the FP32 paths'
               2e-5 of the oracle's FP64 paths
  sweep        on its own binary16 paths: the replay check (every date's
               normal equations and the price within the FP32 bounds of the
               kernel's arithmetic, tests/lsm_replay.py), and within 2e-4 K
               of the oracle's sweep on the same paths
  price        within 2e-4 K of the oracle on the unrounded points (the
               single options of 2^14 and 2^20 paths, a 1 % sample of the
               4096-option batch); an option whose oracle price itself moves
               by more than half that under binary16 rounding of its paths
               is held to the replay check instead (check_mixed16_vs_oracle)
  batch        equal to the option priced alone, bit for bit
"""
import numpy as np
import pytest

import oracle
import workloads
from lsm_replay import gpu_fit, gpu_replay, replay_check
from lsm_sensitivity import binary16_moneyness, check_mixed16_vs_oracle

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


def _ulp16(y):
    """Spacing of binary16 numbers at |y| (subnormal spacing 2^-24 below 2^-14)."""
    e = np.floor(np.log2(np.maximum(np.abs(y), 2.0 ** -14)))
    return 2.0 ** (e - 10)


def _ulp32(v):
    """Spacing of FP32 numbers at |v| (at least 2^-126)."""
    e = np.floor(np.log2(np.maximum(np.abs(v), 2.0 ** -126)))
    return 2.0 ** (e - 23)


def _gpu_price(amc, ctx, o, prec):
    return amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                  o.rule, prec)


def _oracle_price(o):
    return oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type, seed=o.seed,
                        rule=o.rule)


PATH_CASES = [
    ("ls_table1", workloads.single_small()),
    ("call_ragged", workloads.Option(110.0, 100.0, 0.03, 0.45, 2.0, 37, 3001, basis=3, type=1, seed=9)),
    ("max_dates", workloads.Option(100.0, 90.0, 0.05, 0.2, 1.0, 512, 700, basis=3, seed=16)),
    ("one_date", workloads.Option(100.0, 100.0, 0.05, 0.3, 0.5, 1, 2048, basis=2, seed=5)),
    ("huge_vol", workloads.Option(100.0, 100.0, 0.05, 1.5, 1.0, 50, 8192, basis=4, seed=21)),
]


@pytest.mark.parametrize("name,o", PATH_CASES, ids=[c[0] for c in PATH_CASES])
def test_binary16_paths_are_the_fp32_paths_rounded(amc, ctx, torch, name, o):
    ld = amc.amc_path_ld(o.n_paths)
    S32 = torch.full((o.n_steps, ld), float("nan"), dtype=torch.float32, device="cuda")
    Y16 = torch.full((o.n_steps, ld), float("nan"), dtype=torch.float16, device="cuda")
    amc.amc_generate_paths(ctx, o, amc.AMC_MIXED, S32)
    amc.amc_generate_paths(ctx, o, amc.AMC_MIXED16, Y16)
    torch.cuda.synchronize()
    S = S32[:, :o.n_paths].double().cpu().numpy()
    y32 = S / o.K - 1.0
    y16 = Y16[:, :o.n_paths].double().cpu().numpy()
    assert np.isfinite(y16).all()
    # both are 2^e of an FP32 exponent e (the spot, or spot over strike, folded
    # into it) less 1 for y: each carries ln 2 times the rounding of its own e
    # (half an FP32 ulp of e, twice: the drift and the FMA) and the rounding
    # of 2^e; then y16 rounds once more to binary16
    u = 2.0 ** -24
    rel = np.log(2.0) * (_ulp32(np.log2(S)) + _ulp32(np.log2(S / o.K))) + 8 * u
    dev = np.abs(y16 - y32) - (_ulp16(y32) + rel * (1.0 + np.abs(y32)))
    assert dev.max() <= 0.0, (name, np.unravel_index(dev.argmax(), dev.shape), dev.max())
    # and against the oracle's FP64 paths: the FP32 paths' 2e-5 on top
    y64 = oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed) / o.K - 1.0
    dev = np.abs(y16 - y64) - (_ulp16(y64) + 2e-5 * (1.0 + y64))
    assert dev.max() <= 0.0, (name, dev.max())


def test_binary16_paths_full_size_sampled(amc, ctx, torch):
    """2^20 paths x 252 dates: sampled column blocks against the oracle's
    paths of the same points."""
    o = workloads.single_large()
    ld = amc.amc_path_ld(o.n_paths)
    Y16 = torch.empty((o.n_steps, ld), dtype=torch.float16, device="cuda")
    amc.amc_generate_paths(ctx, o, amc.AMC_MIXED16, Y16)
    torch.cuda.synchronize()
    for first in (0, 12345, o.n_paths - 700):
        y16 = Y16[:, first:first + 700].double().cpu().numpy()
        y64 = oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, 700, o.seed, first=first) / o.K - 1.0
        dev = np.abs(y16 - y64) - (_ulp16(y64) + 2e-5 * (1.0 + y64))
        assert dev.max() <= 0.0, (first, dev.max())


SWEEP_CASES = [
    ("ls_table1", workloads.single_small(), False),
    ("cluster_4ctas", workloads.Option(100.0, 95.0, 0.04, 0.35, 1.5, 90, 50000 + 17, basis=4, seed=31), False),
    ("l2_exchange", workloads.scaled(workloads.single_large(), n_paths=2 ** 18 + 2 ** 17 + 3, n_steps=64), False),
    ("call_p3", workloads.Option(95.0, 100.0, 0.02, 0.25, 1.0, 40, 20000, basis=3, type=1, seed=32), False),
    ("two_dates_p1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 2, 1000, basis=1, seed=14), False),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18), False),
    ("streaming", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 40000 + 3, basis=3, seed=33), True),
    ("streaming_call", workloads.Option(100.0, 95.0, 0.03, 0.3, 1.0, 30, 30000, basis=4, type=1, seed=34), True),
]


@pytest.mark.parametrize("name,o,streaming", SWEEP_CASES, ids=[c[0] for c in SWEEP_CASES])
def test_binary16_sweep_on_its_own_paths(amc, ctx, torch, name, o, streaming):
    Sh, coef, got = gpu_fit(amc, ctx, torch, o, streaming=streaming, h16=True)
    d = replay_check(Sh, o, coef, got)
    assert d["residual_ratio"] <= 1.0 and d["price_ratio"] <= 1.0, (name, d)
    ref = oracle.lsm(Sh, o.type, o.K, o.r, o.T, o.basis)
    assert abs(got["price"] - ref["price"]) <= 2e-4 * o.K, (name, got, ref)
    assert got["degenerate_dates"] == ref["degenerate_dates"]


@pytest.mark.parametrize("name,o", [("config1_ls_table1", workloads.single_small()),
                                    ("config2_2p20x252", workloads.single_large())],
                         ids=["config1", "config2"])
def test_binary16_price_vs_oracle(amc, ctx, name, o):
    ref = _oracle_price(o)
    got = _gpu_price(amc, ctx, o, amc.AMC_MIXED16)
    assert got["status"] == 0
    assert abs(got["price"] - ref["price"]) <= 2e-4 * o.K, (name, got, ref)
    assert got["degenerate_dates"] == ref["degenerate_dates"]


def test_binary16_oracle_on_rounded_points_is_within_the_bar(amc, ctx):
    """The oracle's own price on its points rounded to binary16 moneyness
    (no GPU arithmetic), against the GPU's AMC_MIXED16 price: the rounding
    is the only change of the points, so the two agree to 2e-4 K on a stable
    option."""
    o = workloads.scaled(workloads.single_large(), n_paths=2 ** 16)
    S = oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed)
    ref = oracle.lsm(binary16_moneyness(S, o.K), o.type, o.K, o.r, o.T, o.basis)["price"]
    got = _gpu_price(amc, ctx, o, amc.AMC_MIXED16)["price"]
    assert abs(got - ref) <= 2e-4 * o.K, (got, ref)


def test_binary16_batch_sampled_vs_oracle_and_alone(amc, ctx):
    """Config 3 (the 4096-option batch, 2^14..2^18 paths, 12..365 dates) in
    AMC_MIXED16: a seeded sample equals the option priced alone bit for bit,
    and a seeded 1 % sample is within 2e-4 K of the oracle on the unrounded
    points (check_mixed16_vs_oracle for the options that binary16 rounding
    itself moves beyond the bar)."""
    opts = workloads.batch_options()
    res = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED16)
    assert all(r["status"] == 0 for r in res)
    for i in np.random.default_rng(46).choice(len(opts), size=8, replace=False):
        s = _gpu_price(amc, ctx, opts[i], amc.AMC_MIXED16)
        assert res[i]["price"] == s["price"] and res[i]["std_err"] == s["std_err"], (i, res[i], s)
    for i in np.random.default_rng(44).choice(len(opts), size=len(opts) // 100, replace=False):
        o = opts[i]
        ref = _oracle_price(o)
        check_mixed16_vs_oracle(o, res[i]["price"], ref["price"],
                                lambda: _gpu_price(amc, ctx, o, amc.AMC_FP64)["price"],
                                lambda: gpu_replay(amc, ctx, o, h16=True))
        assert res[i]["degenerate_dates"] == ref["degenerate_dates"], (i, res[i], ref)


def test_binary16_batch_device_form_equals_host_form(amc, ctx, torch):
    opts = [workloads.scaled(o, n_paths=min(o.n_paths, 2 ** 15)) for o in workloads.batch_options(n=24)]
    host = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED16)
    res = torch.full((len(opts), amc.AMC_RES_DOUBLES), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    amc.amc_price_batch_device(ctx, opts, res, amc.AMC_MIXED16, stream=st)
    st.synchronize()
    got = res.cpu().numpy()
    for i, h in enumerate(host):
        assert got[i][0] == h["price"] and got[i][1] == h["std_err"], (i, got[i], h)


def test_binary16_is_refused_where_it_is_not_read(amc, ctx, torch):
    """Greeks, the pathwise rules, the boundary valuation, the fused and
    dual calls, serving and the allocation-free sweep take no binary16 path
    array: AMC_EINVAL before any device work."""
    o = workloads.single_small()
    ld = amc.amc_path_ld(o.n_paths)
    Y = torch.zeros((o.n_steps, ld), dtype=torch.float16, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    coef = torch.zeros((o.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    paper = workloads.Option(**{**o.as_dict(), "rule": workloads.RULE_PAPER_UB})
    calls = [
        lambda: amc.amc_sweep(ctx, o, amc.AMC_MIXED16, Y, res, with_greeks=True),
        lambda: amc.amc_sweep(ctx, paper, amc.AMC_MIXED16, Y, res),
        lambda: amc.amc_value_boundary(ctx, o, amc.AMC_MIXED16, Y, coef, res),
        lambda: amc.amc_price_fused(ctx, o, amc.AMC_MIXED16, res, coef),
        lambda: amc.amc_generate_paths_permuted(ctx, o, amc.AMC_MIXED16, Y),
        lambda: amc.amc_greeks(ctx, [o], amc.AMC_MIXED16),
        lambda: amc.amc_price_batch(ctx, [o, paper], amc.AMC_MIXED16),
        lambda: amc.amc_sweep_noalloc(o, amc.AMC_MIXED16, Y, res),
        lambda: amc.amc_serve_start(ctx, prec=amc.AMC_MIXED16),
    ]
    for k, call in enumerate(calls):
        with pytest.raises(amc.AmcError) as ei:
            call()
        assert ei.value.code == amc.AMC_EINVAL, k
    torch.cuda.synchronize()
    assert torch.count_nonzero(res).item() == 0 and torch.count_nonzero(Y).item() == 0
