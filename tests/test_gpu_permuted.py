"""The paper's randomisation (LCG permutation of each dimension's unshifted
quasi-random points) on the GPU vs the FP64 oracle, through the C ABI.

Bars: paths rtol 1e-11 (FP64) / 2e-5 (mixed), as for the digitally shifted
paths; LSM prices on the permuted points |dP| <= 2e-4 K with equal
degenerate counts; over independent seeds the permuted estimator agrees with
the digitally shifted one within the error of the mean."""
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
    c = amc.Context(0, arena_bytes=4 << 30)
    yield c
    c.close()


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _perm_paths(amc, ctx, torch, opt, prec):
    ld = amc.amc_path_ld(opt.n_paths)
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.full((opt.n_steps, ld), float("nan"), dtype=dt, device="cuda")
    amc.amc_generate_paths_permuted(ctx, opt, prec, S)
    torch.cuda.synchronize()
    return S


CASES = [(16, 4096, 9), (50, 12345, 3), (252, 3000, 5), (7, 1, 2), (1, 333, 4), (365, 777, 6)]


@pytest.mark.parametrize("m,n,seed", CASES)
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_permuted_paths_vs_oracle(amc, ctx, torch, m, n, seed, prec):
    opt = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, m, n, basis=3, seed=seed)
    S = _perm_paths(amc, ctx, torch, opt, prec)[:, :n].double().cpu().numpy()
    ref = oracle.paths_permuted(opt.S0, opt.r, opt.sigma, opt.T, m, n, seed)
    tol = 1e-11 if prec == amc.AMC_FP64 else 2e-5
    np.testing.assert_allclose(S, ref, rtol=tol)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_lsm_on_permuted_points_vs_oracle(amc, ctx, torch, prec):
    for opt in (workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=1),
                workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 100, 30001, basis=4, seed=12),
                workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11)):
        S = _perm_paths(amc, ctx, torch, opt, prec)
        res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
        amc.amc_sweep(ctx, opt, prec, S, res)
        got = amc.res_to_dict(res.cpu().numpy())
        Sr = oracle.paths_permuted(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed)
        ref = oracle.lsm(Sr, opt.type, opt.K, opt.r, opt.T, opt.basis)
        assert got["status"] == 0
        assert abs(got["price"] - ref["price"]) <= 2e-4 * opt.K, (opt, got, ref)
        assert got["degenerate_dates"] == ref["degenerate_dates"]


def test_permuted_and_shifted_estimators_agree_over_seeds(amc, ctx, torch):
    base = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=0)
    perm, shift = [], []
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    for s in range(12):
        opt = workloads.Option(**{**base.as_dict(), "seed": 100 + s})
        S = _perm_paths(amc, ctx, torch, opt, amc.AMC_MIXED)
        amc.amc_sweep(ctx, opt, amc.AMC_MIXED, S, res)
        perm.append(float(res[0].item()))
    shift = [r["price"] for r in amc.amc_price_batch(ctx, [workloads.Option(**{**base.as_dict(), "seed": 100 + s})
                                                            for s in range(12)], amc.AMC_MIXED)]
    se = np.sqrt(np.var(perm, ddof=1) / len(perm) + np.var(shift, ddof=1) / len(shift))
    assert abs(np.mean(perm) - np.mean(shift)) < 4 * se + 1e-3
