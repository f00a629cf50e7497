"""Steps 1-4 without a path array (amc_price_fused) on the GPU vs the FP64
oracle and vs the stored-path kernels, through the C ABI.

Bars: against the oracle on identical points, |dP| <= 2e-4 K (mixed) and
1e-10 K (FP64); against generating, storing and sweeping the same paths,
5e-6 K (mixed: the same FP32 paths and decisions, but the stored-path
kernels discount by repeated products of the FP32 e^{-r dt}, a systematic
relative error of up to d 2^-25 after d dates, about 1.5e-6 K at 365 dates,
where the fused kernel takes e^{-r t_d} directly; sums in another order)
and 1e-12 K (FP64).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


@pytest.fixture(scope="module")
def ctx(amc):
    c = amc.Context(0, arena_bytes=8 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _fused(amc, ctx, torch, opt, prec, coef=None):
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_price_fused(ctx, opt, prec, res, coef)
    torch.cuda.synchronize()
    return amc.res_to_dict(res.cpu().numpy())


def _stored(amc, ctx, opt, prec):
    return amc.amc_price_american(ctx, opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.basis,
                                  opt.type, opt.seed, opt.rule, prec)


def _oracle(opt):
    return oracle.price(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, basis=opt.basis,
                        type=opt.type, seed=opt.seed, rule=opt.rule)


PW = workloads.RULE_PAPER_UB
EU = workloads.RULE_EUROPEAN
CASES = [
    ("ls_table1_paper", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, seed=1, rule=PW)),
    ("one_date_paper", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=3, rule=PW)),
    ("two_dates_paper", workloads.Option(100.0, 95.0, 0.03, 0.3, 0.5, 2, 777, seed=4, rule=PW)),
    ("ragged_call_paper", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, type=1, seed=11, rule=PW)),
    ("many_dates_paper", workloads.Option(100.0, 110.0, 0.02, 0.4, 2.0, 365, 8192, seed=15, rule=PW)),
    ("ls_table1_european", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, seed=1, rule=EU)),
    ("ragged_call_european", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, type=1, seed=11, rule=EU)),
    ("one_date_european", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 5, seed=3, rule=EU)),
    ("max_dates_paper", workloads.Option(100.0, 100.0, 0.05, 0.3, 2.0, 512, 3000, seed=16, rule=PW)),
]


@pytest.mark.parametrize("name,opt", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_fused_price_vs_oracle_and_stored(amc, ctx, torch, name, opt, prec):
    got = _fused(amc, ctx, torch, opt, prec)
    ref = _oracle(opt)
    st = _stored(amc, ctx, opt, prec)
    assert got["status"] == 0 and got["degenerate_dates"] == 0
    tol = 1e-10 if prec == amc.AMC_FP64 else 2e-4
    assert abs(got["price"] - ref["price"]) <= tol * opt.K, (got, ref)
    assert abs(got["std_err"] - ref["std_err"]) <= 1e-3 * ref["std_err"] + tol * opt.K
    same = 1e-12 if prec == amc.AMC_FP64 else 5e-6
    assert abs(got["price"] - st["price"]) <= same * opt.K, (got, st)


@pytest.mark.parametrize("rule", [PW, EU], ids=["paper", "european"])
def test_fused_full_size_vs_oracle(amc, ctx, torch, rule):
    opt = workloads.Option(**{**workloads.single_large().as_dict(), "rule": rule})
    got = _fused(amc, ctx, torch, opt, amc.AMC_MIXED)
    ref = _oracle(opt)
    assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (got, ref)
    assert abs(got["price"] - _stored(amc, ctx, opt, amc.AMC_MIXED)["price"]) <= 5e-6 * opt.K


BOUNDARY_CASES = [
    ("ls_table1", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=1)),
    ("ragged_call_p2", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11)),
    ("ragged_put_p4", workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 100, 30001, basis=4, seed=12)),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18)),
    ("one_date", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=13)),
    ("max_dates", workloads.Option(100.0, 100.0, 0.05, 0.3, 2.0, 512, 3000, basis=4, seed=17)),
]


@pytest.mark.parametrize("name,opt", BOUNDARY_CASES, ids=[c[0] for c in BOUNDARY_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_fused_boundary_valuation_vs_oracle_and_stored(amc, ctx, torch, name, opt, prec):
    """The oracle's own boundary (fitted on the option's points) applied to
    the points of another seed, fused vs the oracle's valuation and vs the
    valuation kernel on stored paths."""
    fit = oracle.lsm(oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed), opt.type,
                     opt.K, opt.r, opt.T, opt.basis, details=True)
    vopt = workloads.Option(**{**opt.as_dict(), "seed": opt.seed + 100})
    Sv = oracle.paths(vopt.S0, vopt.r, vopt.sigma, vopt.T, vopt.n_steps, vopt.n_paths, vopt.seed)
    want = oracle.value_boundary(Sv, vopt.type, vopt.K, vopt.r, vopt.T, fit["beta"], fit["deg"])
    c = np.zeros((opt.n_steps, amc.AMC_COEF_STRIDE))
    c[:, :opt.basis] = fit["beta"] / opt.K
    c[:, 4] = fit["deg"]
    coef = torch.tensor(c, dtype=torch.float64, device="cuda")
    got = _fused(amc, ctx, torch, vopt, prec, coef)
    tol = 1e-10 if prec == amc.AMC_FP64 else 2e-4
    assert got["status"] == 0
    assert abs(got["price"] - want["price"]) <= tol * opt.K, (got, want)
    assert got["degenerate_dates"] == want["degenerate_dates"]
    ld = amc.amc_path_ld(vopt.n_paths)
    S = torch.empty((vopt.n_steps, ld), dtype=torch.float64 if prec == amc.AMC_FP64 else torch.float32,
                    device="cuda")
    amc.amc_generate_paths(ctx, vopt, prec, S)
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_value_boundary(ctx, vopt, prec, S, coef, res)
    torch.cuda.synchronize()
    st = amc.res_to_dict(res.cpu().numpy())
    same = 1e-12 if prec == amc.AMC_FP64 else 5e-6
    assert abs(got["price"] - st["price"]) <= same * opt.K, (got, st)


def test_fused_is_deterministic(amc, ctx, torch):
    opt = CASES[0][1]
    a = _fused(amc, ctx, torch, opt, amc.AMC_MIXED)
    b = _fused(amc, ctx, torch, opt, amc.AMC_MIXED)
    assert a == b


def test_fused_rejects_bad_arguments(amc, ctx, torch):
    opt = CASES[0][1]
    lsm = workloads.Option(**{**opt.as_dict(), "rule": workloads.RULE_LSM})
    coef = torch.zeros((opt.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    for o, c in ((opt, coef), (lsm, None)):          # a boundary for a rule without one; LSM without one
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_price_fused(ctx, o, amc.AMC_MIXED, res, c)
        assert ei.value.code == amc.AMC_EINVAL
