"""Second Longstaff-Schwartz pass (out-of-sample valuation) on the GPU vs the
FP64 oracle, through the C ABI.

Bars:
  fitted boundary       degenerate flags equal; continuation value c(y) at the
                        5..95 % quantiles of the date's in-the-money moneyness
                        (a regression is only determined on its data) within
                        1e-9 K (FP64) / 5e-3 K (mixed: the FP32 moment sums
                        carry relative errors ~1e-6, which the equilibrated
                        Gram matrix of a cubic on clustered moneyness, with
                        condition numbers up to ~1e4, amplifies to a few 1e-3
                        of c ~ 0.5); the price bars below are the binding ones
  valuation, same coefficients and points   |dP| <= 2e-4 K (FP64: 1e-10 K)
  valuation on the fitting paths            = in-sample price (1e-6 K: only
                                              the order of the final sums differs)
  out-of-sample price   |dP| <= 2e-4 K on identical points (the mixed in-sample
                        fit of an option that is unstable at FP32 precision:
                        the replay check and the FP64 price instead,
                        check_mixed_vs_oracle)
"""
import numpy as np
import pytest

import oracle
import workloads
from lsm_replay import gpu_replay
from lsm_sensitivity import check_mixed_vs_oracle, fp32_noise_spread

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


def _dev_paths(amc, ctx, torch, opt, prec):
    ld = amc.amc_path_ld(opt.n_paths)
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.empty((opt.n_steps, ld), dtype=dt, device="cuda")
    amc.amc_generate_paths(ctx, opt, prec, S)
    return S


def _fit(amc, ctx, torch, opt, prec):
    S = _dev_paths(amc, ctx, torch, opt, prec)
    coef = torch.full((opt.n_steps, amc.AMC_COEF_STRIDE), float("nan"), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_fit_boundary(ctx, opt, prec, S, coef, res)
    torch.cuda.synchronize()
    return S, coef, amc.res_to_dict(res.cpu().numpy())


def _value(amc, ctx, torch, opt, prec, S, coef):
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_value_boundary(ctx, opt, prec, S, coef, res)
    torch.cuda.synchronize()
    return amc.res_to_dict(res.cpu().numpy())


def _oracle_fit(opt, with_paths=False):
    S = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    res = oracle.lsm(S, opt.type, opt.K, opt.r, opt.T, opt.basis, details=True)
    return (res, S) if with_paths else res


FIT_CASES = [
    ("ls_table1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=1)),
    ("ragged_call_p2", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11)),
    ("ragged_put_p4", workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 100, 30001, basis=4, seed=12)),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18)),
    ("one_date", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=13)),
]


@pytest.mark.parametrize("name,opt", FIT_CASES, ids=[c[0] for c in FIT_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_fitted_boundary_vs_oracle(amc, ctx, torch, name, opt, prec):
    _, coef, fit = _fit(amc, ctx, torch, opt, prec)
    ref, Sref = _oracle_fit(opt, with_paths=True)
    c = coef.cpu().numpy()
    m, p = opt.n_steps, opt.basis
    assert np.all(np.isfinite(c))
    deg_gpu = (c[:, 4] != 0).astype(np.int32)
    np.testing.assert_array_equal(deg_gpu, ref["deg"])
    assert fit["degenerate_dates"] == ref["degenerate_dates"]
    assert np.all(c[:, p:4] == 0.0)
    tol = 1e-9 if prec == amc.AMC_FP64 else 5e-3
    for j in range(m - 1):
        if ref["deg"][j]:
            assert np.all(c[j, :4] == 0.0)
            continue
        yj = Sref[j] / opt.K - 1.0
        yj = yj[yj < 0] if opt.type == oracle.PUT else yj[yj > 0]
        V = np.vander(np.quantile(yj, np.linspace(0.05, 0.95, 19)), p, increasing=True)
        got = V @ c[j, :p]
        want = V @ (ref["beta"][j] / opt.K)
        assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want))), (j, got, want)


@pytest.mark.parametrize("name,opt", FIT_CASES, ids=[c[0] for c in FIT_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_valuation_with_the_oracle_boundary_vs_oracle(amc, ctx, torch, name, opt, prec):
    """Same coefficients (the oracle's), same points: only the kernel and the
    path precision differ."""
    ref = _oracle_fit(opt)
    vopt = workloads.Option(**{**opt.as_dict(), "seed": opt.seed + 100})
    Sv = oracle.paths(vopt.S0, vopt.r, vopt.sigma, vopt.T, vopt.n_steps, vopt.n_paths, vopt.seed)
    want = oracle.value_boundary(Sv, vopt.type, vopt.K, vopt.r, vopt.T, ref["beta"], ref["deg"])
    c = np.zeros((opt.n_steps, amc.AMC_COEF_STRIDE))
    c[:, :opt.basis] = ref["beta"] / opt.K
    c[:, 4] = ref["deg"]
    coef = torch.tensor(c, dtype=torch.float64, device="cuda")
    S = _dev_paths(amc, ctx, torch, vopt, prec)
    got = _value(amc, ctx, torch, vopt, prec, S, coef)
    tol = 1e-10 if prec == amc.AMC_FP64 else 2e-4
    assert got["status"] == 0
    assert abs(got["price"] - want["price"]) <= tol * opt.K, (got, want)
    assert abs(got["std_err"] - want["std_err"]) <= 1e-3 * want["std_err"] + tol * opt.K
    assert got["degenerate_dates"] == want["degenerate_dates"]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_valuation_on_the_fitting_paths_repeats_the_in_sample_price(amc, ctx, torch, prec):
    for opt in (FIT_CASES[0][1], FIT_CASES[2][1], workloads.scaled(workloads.single_large(), n_paths=2 ** 18)):
        S, coef, fit = _fit(amc, ctx, torch, opt, prec)
        val = _value(amc, ctx, torch, opt, prec, S, coef)
        assert val["status"] == 0 and fit["status"] == 0
        assert abs(val["price"] - fit["price"]) <= 1e-6 * opt.K, (opt, fit, val)
        assert val["degenerate_dates"] == fit["degenerate_dates"]


OOS_CASES = FIT_CASES + [
    ("many_dates", workloads.Option(100.0, 110.0, 0.02, 0.4, 2.0, 365, 8192, basis=3, seed=15)),
    ("big_group", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 60, 2 ** 19 + 3, basis=4, seed=19)),
]


@pytest.mark.parametrize("name,opt", OOS_CASES, ids=[c[0] for c in OOS_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_out_of_sample_price_vs_oracle(amc, ctx, torch, name, opt, prec):
    vseed = opt.seed + 1000
    fit, val = amc.amc_price_oos(ctx, opt, vseed, prec)
    rfit, rval = oracle.price_oos(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths,
                                  basis=opt.basis, type=opt.type, seed=opt.seed, value_seed=vseed)
    assert fit["status"] == 0 and val["status"] == 0
    if prec == amc.AMC_MIXED:
        # the 365-date put on 8192 paths is unstable at FP32 precision (its oracle
        # price moves 2.7e-4 K under 2e-5 path noise and 1.2e-4 K under FP32
        # sums): the in-sample fit is held to 2e-4 K unless the oracle shows that,
        # and then to the replay check and the FP64 price
        check_mixed_vs_oracle(opt, fit["price"], rfit["price"], lambda: amc.amc_price_oos(ctx, opt, vseed, 0)[0]["price"],
                              lambda: gpu_replay(amc, ctx, opt))
    else:
        assert abs(fit["price"] - rfit["price"]) <= 2e-4 * opt.K
    if prec == amc.AMC_MIXED and abs(val["price"] - rval["price"]) > 2e-4 * opt.K:
        # the value out of sample depends on the fitted boundary; on an option
        # whose fit is unstable at FP32 precision (the oracle shows it) the
        # valuation is held to the oracle's valuation under the GPU's own
        # fitted boundary (the same one: the fit is deterministic)
        assert fp32_noise_spread(opt) > 1e-4, ("out-of-sample value off the oracle on an FP32-stable option", val, rval)
        _, coef, _ = _fit(amc, ctx, torch, opt, prec)
        c = coef.cpu().numpy()
        Sv = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, vseed)
        want = oracle.value_boundary(Sv, opt.type, opt.K, opt.r, opt.T, c[:, :opt.basis] * opt.K,
                                     (c[:, 4] != 0).astype(np.int32))
        assert abs(val["price"] - want["price"]) <= 2e-4 * opt.K, (val, want)
    else:
        assert abs(val["price"] - rval["price"]) <= 2e-4 * opt.K, (val, rval)
        assert val["degenerate_dates"] == rval["degenerate_dates"]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_out_of_sample_full_size_vs_oracle(amc, ctx, prec):
    opt = workloads.single_large()
    fit, val = amc.amc_price_oos(ctx, opt, 7, prec)
    rfit, rval = oracle.price_oos(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths,
                                  basis=opt.basis, type=opt.type, seed=opt.seed, value_seed=7)
    assert abs(fit["price"] - rfit["price"]) <= 2e-4 * opt.K
    assert abs(val["price"] - rval["price"]) <= 2e-4 * opt.K
    # low-biased against the in-sample estimate, within the error bars of both
    assert val["price"] <= fit["price"] + 3 * (fit["std_err"] + val["std_err"])


def test_boundary_calls_reject_bad_arguments(amc, ctx, torch):
    opt = workloads.single_small()
    S = _dev_paths(amc, ctx, torch, opt, amc.AMC_MIXED)
    coef = torch.zeros((opt.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    euro = workloads.Option(**{**opt.as_dict(), "rule": 2})
    for call in (amc.amc_fit_boundary, amc.amc_value_boundary):
        with pytest.raises(amc.AmcError) as ei:
            call(ctx, euro, amc.AMC_MIXED, S, coef, res)
        assert ei.value.code == amc.AMC_EINVAL
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_price_oos(ctx, euro, 3, amc.AMC_MIXED)
    assert ei.value.code == amc.AMC_EINVAL
