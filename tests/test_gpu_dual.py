"""Dual upper bound of a fitted boundary on the GPU vs the FP64 oracle,
through the C ABI.

The boundary is the oracle's own (coefficients and degenerate flags of an
oracle LSM fit), so that only the dual computation differs.  Bars:
  AMC_FP64   per-path U within 1e-9 K, mean U and L0 within 1e-10 K: same
             normals (the same counter-based SplitMix64 stream, FP64 inverse
             normal), the same GBM steps; only rounding order differs
  AMC_MIXED  mean U and L0 within 2e-4 K.  FP32 inner paths move an inner
             stopping decision where FP64 h - c is within ~1e-6 K of zero;
             each such flip changes one inner payoff out of n_in, and the
             changes are of either sign, so per-path values move but the
             mean over the outer paths stays inside the price bar
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


def _dev_paths(amc, ctx, torch, opt, prec):
    ld = amc.amc_path_ld(opt.n_paths)
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.empty((opt.n_steps, ld), dtype=dt, device="cuda")
    amc.amc_generate_paths(ctx, opt, prec, S)
    return S


def _coef(amc, torch, opt, beta, deg):
    c = np.zeros((opt.n_steps, amc.AMC_COEF_STRIDE))
    c[:, :opt.basis] = beta / opt.K
    c[:, 4] = deg
    return torch.tensor(c, dtype=torch.float64, device="cuda")


def _gpu_dual(amc, ctx, torch, opt, prec, coef, n_in, seed_in):
    S = _dev_paths(amc, ctx, torch, opt, prec)
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    U = torch.empty(opt.n_paths, dtype=torch.float64, device="cuda")
    amc.amc_dual_upper(ctx, opt, prec, S, coef, n_in, seed_in, res, U)
    torch.cuda.synchronize()
    return res.cpu().numpy(), U.cpu().numpy()


def _oracle_boundary(opt, n_fit, fit_seed):
    fit = oracle.lsm(oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, n_fit, fit_seed), opt.type, opt.K,
                     opt.r, opt.T, opt.basis, details=True)
    return fit["beta"], fit["deg"]


# (name, outer option (n_paths outer paths, seed = outer seed), fitting paths, fitting seed, inner paths)
DUAL_CASES = [
    ("ls_put_m10", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 1000, basis=3, seed=31), 2 ** 13, 1, 64),
    ("ragged_call_p2", workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 333, basis=2, type=1, seed=32), 12345, 2,
     37),
    ("put_p4_m24", workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 24, 517, basis=4, seed=33), 30001, 3, 50),
    ("deep_otm_degenerate", workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 300, basis=3, seed=34), 2000, 4, 32),
    ("one_date", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 4096, seed=35), 4096, 5, 8),
    ("many_warps_few_lanes", workloads.Option(100.0, 100.0, 0.05, 0.3, 1.0, 40, 129, basis=3, seed=36), 8192, 6, 5),
    ("max_dates", workloads.Option(100.0, 100.0, 0.05, 0.3, 2.0, 512, 40, basis=4, seed=37), 8192, 7, 4),
]


# The 512-date case (the largest shared-memory layout) is held to the FP64
# bars only: each outer path takes about 1e5 FP32 stopping decisions there,
# so a few land within the FP32 error of the boundary, and with 4 inner paths
# each such flip moves a continuation estimate by a quarter of a payoff; the
# mean over 40 outer paths then moves by far more than 2e-4 K.
FP64_ONLY = {"max_dates"}


@pytest.mark.parametrize("name,opt,n_fit,fit_seed,n_in", DUAL_CASES, ids=[c[0] for c in DUAL_CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_dual_with_the_oracle_boundary_vs_oracle(amc, ctx, torch, name, opt, n_fit, fit_seed, n_in, prec):
    if prec == amc.AMC_MIXED and name in FP64_ONLY:
        pytest.skip("FP32 inner decisions at 512 dates with 4 inner paths: FP64 bars only")
    beta, deg = _oracle_boundary(opt, n_fit, fit_seed)
    seed_in = 1000 + opt.seed
    res, U = _gpu_dual(amc, ctx, torch, opt, prec, _coef(amc, torch, opt, beta, deg), n_in, seed_in)
    So = oracle.paths(opt.S0, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, opt.seed)
    want = oracle.dual_upper(So, opt.type, opt.K, opt.r, opt.sigma, opt.T, beta, deg, n_in, seed_in, details=True)
    assert res[5] == 0
    assert res[4] == int(np.sum(deg[:-1]))
    tol = 1e-10 if prec == amc.AMC_FP64 else 2e-4
    assert abs(res[0] - want["upper"]) <= tol * opt.K, (res, want)
    assert abs(res[6] - want["L0"]) <= tol * opt.K, (res, want)
    assert np.all(np.isfinite(U))
    np.testing.assert_allclose(np.mean(U), res[0], rtol=0, atol=1e-12 * opt.K)
    if prec == amc.AMC_FP64:
        np.testing.assert_allclose(U, want["U"], rtol=0, atol=1e-9 * opt.K)
        assert res[1] == pytest.approx(want["std_err"], rel=1e-6, abs=1e-12)
    else:
        assert res[1] == pytest.approx(want["std_err"], rel=0.05, abs=1e-4 * opt.K)
    if opt.n_steps == 1:                       # no inner paths: U = L0 = the European estimator
        assert res[7] == 0
        np.testing.assert_allclose(U, res[6], rtol=1e-13)


def test_inner_step_count_with_a_boundary_that_never_exercises(amc, ctx, torch):
    """All dates degenerate: every inner path from t_j runs to t_m, so exactly
    N n_in m (m-1) / 2 steps; U then equals L0 + max_j (Z_j - M_j) with the
    European continuation on every date."""
    opt = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 12, 211, basis=3, seed=41)
    coef = _coef(amc, torch, opt, np.zeros((12, 3)), np.ones(12, dtype=np.int32))
    for prec in (amc.AMC_FP64, amc.AMC_MIXED):
        res, _ = _gpu_dual(amc, ctx, torch, opt, prec, coef, 19, 5)
        assert res[7] == 211 * 19 * 12 * 11 // 2
        assert res[4] == 11


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_dual_is_deterministic_and_the_seed_matters(amc, ctx, torch, prec):
    name, opt, n_fit, fit_seed, n_in = DUAL_CASES[2]
    beta, deg = _oracle_boundary(opt, n_fit, fit_seed)
    coef = _coef(amc, torch, opt, beta, deg)
    r1, U1 = _gpu_dual(amc, ctx, torch, opt, prec, coef, n_in, 77)
    r2, U2 = _gpu_dual(amc, ctx, torch, opt, prec, coef, n_in, 77)
    r3, _ = _gpu_dual(amc, ctx, torch, opt, prec, coef, n_in, 78)
    assert np.array_equal(r1, r2) and np.array_equal(U1, U2)
    assert r3[0] != r1[0]
    assert abs(r3[0] - r1[0]) < 5 * (r1[1] + r3[1])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_price_dual_vs_oracle(amc, ctx, prec):
    opt = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 2 ** 13, basis=3, seed=1)
    fit, low, up = amc.amc_price_dual(ctx, opt, 2, 1024, 64, 3, prec)
    rfit, rlow, rup = oracle.price_dual(opt.S0, opt.K, opt.r, opt.sigma, opt.T, opt.n_steps, opt.n_paths, 1024, 64,
                                        basis=opt.basis, type=opt.type, seed=opt.seed, outer_seed=2, seed_in=3)
    tol = 1e-8 if prec == amc.AMC_FP64 else 2e-4
    assert fit["status"] == low["status"] == up["status"] == 0
    assert abs(fit["price"] - rfit["price"]) <= tol * opt.K
    assert abs(low["price"] - rlow["price"]) <= tol * opt.K
    assert abs(up["price"] - rup["upper"]) <= tol * opt.K, (up, rup)


def test_bounds_bracket_the_bermudan_tree(amc, ctx):
    """Lower (boundary applied to independent paths) and dual upper bound
    around the Bermudan binomial value.  The upper bound's excess over the
    value is mostly inner-sampling bias (the maximum over dates of noisy
    martingale increments): it falls as the inner paths grow (0.28, 0.10,
    0.04 over the tree at 64, 256, 1024 inner paths in the oracle on 512
    outer paths), and at 1024 inner paths the bound is within 1.5 % of the
    tree."""
    opt = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 16, basis=3, seed=1)
    tree = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, 50, bermudan=True)
    ups = []
    for n_in in (64, 256, 1024):
        fit, low, up = amc.amc_price_dual(ctx, opt, 9, 4096, n_in, 10, amc.AMC_MIXED)
        assert low["price"] <= tree + 3 * low["std_err"]
        assert up["price"] >= tree - 3 * up["std_err"]
        ups.append(up["price"])
    excess = [u - tree for u in ups]
    assert excess[1] < 0.6 * excess[0] and excess[2] < 0.6 * excess[1], excess
    assert excess[2] < 0.015 * tree, excess


def test_dual_full_size_sampled_vs_oracle(amc, ctx, torch):
    """The 2^20-path, 252-date put's boundary (GPU fit), dual on 4096 outer
    paths with 128 inner paths: U(i) - L0 of the first outer paths against
    the oracle on those paths (the inner stream depends only on i, j, k, s),
    as a mean over the sample (mixed arithmetic, see the module bars)."""
    big = workloads.single_large()
    ld = amc.amc_path_ld(big.n_paths)
    S = torch.empty((big.n_steps, ld), dtype=torch.float32, device="cuda")
    amc.amc_generate_paths(ctx, big, amc.AMC_MIXED, S)
    coef = torch.zeros((big.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_fit_boundary(ctx, big, amc.AMC_MIXED, S, coef, res)
    del S
    outer = workloads.Option(**{**big.as_dict(), "n_paths": 4096, "seed": 12})
    gres, U = _gpu_dual(amc, ctx, torch, outer, amc.AMC_MIXED, coef, 128, 13)
    assert gres[5] == 0 and np.all(np.isfinite(U))
    c = coef.cpu().numpy()
    beta, deg = c[:, :big.basis] * big.K, (c[:, 4] != 0).astype(np.int32)
    n_s = 24
    So = oracle.paths(outer.S0, outer.r, outer.sigma, outer.T, outer.n_steps, n_s, outer.seed)
    S_full = oracle.paths(outer.S0, outer.r, outer.sigma, outer.T, outer.n_steps, outer.n_paths, outer.seed)
    np.testing.assert_allclose(So, S_full[:, :n_s], rtol=0, atol=0)
    want = oracle.dual_upper(So, outer.type, outer.K, outer.r, outer.sigma, outer.T, beta, deg, 128, 13, details=True)
    got_v = U[:n_s] - gres[6]
    want_v = want["U"] - want["L0"]
    assert abs(np.mean(got_v - want_v)) <= 2e-4 * big.K, (got_v, want_v)
    assert gres[0] >= gres[6] - 3 * gres[1]


def test_dual_rejects_bad_arguments(amc, ctx, torch):
    opt = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 10, 1000, basis=3, seed=31)
    S = _dev_paths(amc, ctx, torch, opt, amc.AMC_MIXED)
    coef = torch.zeros((opt.n_steps, amc.AMC_COEF_STRIDE), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    bad = [
        (opt, 0),                                                          # no inner paths
        (workloads.Option(**{**opt.as_dict(), "rule": 1}), 8),             # not an LSM boundary
        (opt, amc.AMC_DUAL_MAX_WORK // (1000 * 45) + 1),                   # beyond the work bound
        (workloads.Option(**{**opt.as_dict(), "n_steps": 1, "n_paths": 1}), amc.AMC_DUAL_MAX_INNER + 1),
    ]
    for o, n_in in bad:
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_dual_upper(ctx, o, amc.AMC_MIXED, S, coef, n_in, 1, res)
        assert ei.value.code == amc.AMC_EINVAL
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_price_dual(ctx, workloads.Option(**{**opt.as_dict(), "rule": 2}), 1, 100, 8, 1)
    assert ei.value.code == amc.AMC_EINVAL
