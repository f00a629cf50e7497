"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test ties one oracle function to an independent source: scipy's own
Sobol' and inverse-normal routines, printed worked examples (tests/golden/),
closed forms, invariants of the method, or a second implementation written a
different way (oracle/micro.py).  A dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.micro import lsm_micro

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- SplitMix64
def test_splitmix64_published_outputs():
    g = _golden("splitmix64_seed0.json")
    assert oracle.splitmix64(g["seed"], 3) == [int(h, 16) for h in g["outputs_hex"]]


def test_digital_shift_is_high_word():
    outs = oracle.splitmix64(12345, 7)
    assert list(oracle.shifts(12345, 7)) == [o >> 32 for o in outs]


# ---------------------------------------------------------------- Sobol'
@pytest.mark.parametrize("m", [1, 2, 50, 252, 365, 512])
def test_sobol_bit_exact_vs_scipy(m):
    from scipy.stats import qmc
    n = 1024
    eng = qmc.Sobol(d=m, scramble=False, bits=32)
    ref = np.round(eng.random(n) * 2.0 ** 32).astype(np.uint64).T
    X = oracle.sobol(n, m).astype(np.uint64)
    np.testing.assert_array_equal(X, ref)


def test_sobol_gray_recurrence_equals_direct_formula():
    m = 40
    V = oracle.directions(m)
    rng = np.random.default_rng(0)
    for i0 in [0, 1, 4095, 2 ** 20 - 3, 3 * 2 ** 27 + 11]:
        X = oracle.sobol(9, m, i0=i0, V=V)
        for t in range(9):
            for d in rng.choice(m, 5, replace=False):
                assert X[d, t] == oracle.sobol_direct(V, int(d), i0 + t)


def test_sobol_first_dims_are_textbook():
    V = oracle.directions(3)
    # dim 0: van der Corput; dim 1 (x+1, m1=1): m_k = 1, 3, 5, 15, ... (v_k = m_k/2^k)
    assert [int(v) for v in V[0, :4]] == [1 << 31, 1 << 30, 1 << 29, 1 << 28]
    assert [int(V[1, k]) >> (31 - k) for k in range(5)] == [1, 3, 5, 15, 17]


def test_shifted_points_are_xor():
    X0 = oracle.sobol(64, 10)
    X1 = oracle.sobol(64, 10, seed=7)
    np.testing.assert_array_equal(X1, X0 ^ oracle.shifts(7, 10)[:, None])


# ---------------------------------------------------------------- inverse normal
def test_norm_icdf_vs_scipy_ndtri():
    from scipy.special import ndtri
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.integers(0, 2 ** 32, 4000, dtype=np.uint64),
                         np.array([0, 1, 2, 2 ** 31 - 1, 2 ** 31, 2 ** 32 - 2, 2 ** 32 - 1], dtype=np.uint64)])
    u = oracle.uniform(xs)
    assert np.all((u > 0) & (u < 1))
    z = oracle.norm_icdf(u)
    ref = ndtri(u)
    np.testing.assert_allclose(z, ref, rtol=2e-14, atol=2e-15)


def test_norm_cdf_vs_scipy():
    from scipy.special import ndtr
    x = np.linspace(-9, 9, 1001)
    np.testing.assert_allclose(oracle.norm_cdf(x), ndtr(x), rtol=1e-14, atol=1e-300)


# ---------------------------------------------------------------- Brownian bridge
@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 12, 50, 64, 100, 252, 365])
def test_bridge_covariance_is_min(m):
    T = 1.7
    A = oracle.bridge_matrix(m, T)
    t = np.arange(1, m + 1) * (T / m)
    np.testing.assert_allclose(A @ A.T, np.minimum.outer(t, t), atol=1e-12)


@pytest.mark.parametrize("m", [1, 2, 3, 7, 50, 252, 365])
def test_bridge_schedule_visits_every_date_once(m):
    date, left, right = oracle.bridge_schedule(m)
    assert sorted(date.tolist()) == list(range(1, m + 1))
    assert date[0] == m
    seen = {0, m}
    for k in range(1, m):
        assert left[k] in seen and right[k] in seen and left[k] < date[k] < right[k]
        seen.add(int(date[k]))


@pytest.mark.parametrize("m,date,left,right", [
    (5, [5, 2, 1, 3, 4], [0, 0, 0, 2, 3], [0, 5, 2, 5, 5]),
    (7, [7, 3, 1, 5, 2, 4, 6], [0, 0, 0, 3, 1, 3, 5], [0, 7, 3, 7, 3, 5, 7]),
])
def test_bridge_schedule_worked_examples(m, date, left, right):
    """The bridge reading worked out by hand for dates that are not a power
    of two: W(t_m) first, then the intervals (l, r) split breadth-first, left
    before right, at floor((l + r) / 2), each node conditioned on the ends of
    its interval."""
    d, l, r = oracle.bridge_schedule(m)
    assert (d.tolist(), l.tolist(), r.tolist()) == (date, left, right)


def test_bridge_power_of_two_is_textbook_bisection():
    m = 16
    date, _, _ = oracle.bridge_schedule(m)
    expect = [16, 8, 4, 12, 2, 6, 10, 14, 1, 3, 5, 7, 9, 11, 13, 15]
    assert date.tolist() == expect


# ---------------------------------------------------------------- GBM
def test_gbm_log_space_equals_iterated_eq9():
    S0, r, sigma, T, m = 100.0, 0.05, 0.3, 1.0, 12
    S, W = oracle.paths(S0, r, sigma, T, m, 64, seed=3, with_W=True)
    dt = T / m
    prev, Wprev = np.full(64, S0), np.zeros(64)
    for j in range(m):
        prev = prev * np.exp((r - 0.5 * sigma ** 2) * dt + sigma * (W[j] - Wprev))
        Wprev = W[j]
        np.testing.assert_allclose(S[j], prev, rtol=1e-13)


def test_gbm_martingale_each_date():
    S0, r, sigma, T, m, N = 100.0, 0.05, 0.3, 1.0, 16, 2 ** 14
    S = oracle.paths(S0, r, sigma, T, m, N, seed=11)
    t = np.arange(1, m + 1) * (T / m)
    disc_mean = (np.exp(-r * t)[:, None] * S).mean(axis=1)
    np.testing.assert_allclose(disc_mean, S0, rtol=2e-3)


# ---------------------------------------------------------------- Black-Scholes
def test_bs_textbook_example():
    g = _golden("bs_textbook_example.json")
    c = oracle.bs(oracle.CALL, g["S0"], g["K"], g["r"], g["sigma"], g["T"])
    p = oracle.bs(oracle.PUT, g["S0"], g["K"], g["r"], g["sigma"], g["T"])
    assert abs(c - g["call"]) < g["tol"] and abs(p - g["put"]) < g["tol"]


@pytest.mark.parametrize("S0,K,r,sigma,T", [(36, 40, .06, .2, 1), (100, 100, .05, .3, 1), (90, 110, 0.0, .5, 2)])
def test_bs_put_call_parity(S0, K, r, sigma, T):
    c = oracle.bs(oracle.CALL, S0, K, r, sigma, T)
    p = oracle.bs(oracle.PUT, S0, K, r, sigma, T)
    assert abs((c - p) - (S0 - K * math.exp(-r * T))) < 1e-12


def test_bs_equals_converged_european_tree():
    for tp in (oracle.PUT, oracle.CALL):
        bs = oracle.bs(tp, 36, 40, .06, .2, 1.0)
        tree = oracle.crr(tp, 36, 40, .06, .2, 1.0, 20000, 1, bermudan=True)
        assert abs(bs - tree) < 2e-4


# ---------------------------------------------------------------- CRR tree
def test_crr_american_call_equals_european_call():
    c_am = oracle.crr(oracle.CALL, 100, 100, .05, .3, 1.0, 4000)
    c_eu = oracle.crr(oracle.CALL, 100, 100, .05, .3, 1.0, 4000, 1, bermudan=True)
    assert abs(c_am - c_eu) < 1e-10


def test_crr_ordering_european_bermudan_american():
    eu = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, 1, bermudan=True)
    be = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, 50, bermudan=True)
    am = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000)
    assert eu < be < am
    assert be > 40 - 36 - 1e-12


# ---------------------------------------------------------------- normal equations
def test_solve_normal_matches_lstsq_and_flags_singular():
    rng = np.random.default_rng(5)
    x = rng.uniform(0.3, 1.0, 200)
    y = rng.normal(size=200)
    X = np.vander(x, 4, increasing=True)
    beta = oracle.solve_normal(X.T @ X, X.T @ y)
    ref, *_ = np.linalg.lstsq(X, y, rcond=None)
    np.testing.assert_allclose(beta, ref, rtol=1e-7, atol=1e-9)
    Xs = np.vander(np.full(10, 0.7), 3, increasing=True)       # rank 1
    assert oracle.solve_normal(Xs.T @ Xs, Xs.T @ np.ones(10)) is None


# ---------------------------------------------------------------- LSM
def test_lsm_longstaff_schwartz_worked_example():
    g = _golden("ls2001_example.json")
    S = np.array(g["paths_t1_t2_t3"]).T          # (m=3, N=8) date-major
    res = oracle.lsm(S, oracle.PUT, g["K"], g["r"], g["T"], 3, details=True)
    assert abs(res["price"] - g["value"]) < g["value_tol"]
    K = g["K"]
    # basis in y = S/K - 1  ->  coefficients of 1, S, S^2
    P = np.polynomial.polynomial
    def to_S(b):
        c = np.zeros(3)
        for k in range(3):
            t = P.polypow([-1.0, 1.0 / K], k)
            c[:len(t)] += b[k] * t
        return c
    np.testing.assert_allclose(to_S(res["beta"][1]), g["regression_t2_in_S"], atol=g["coef_tol"])
    np.testing.assert_allclose(to_S(res["beta"][0]), g["regression_t1_in_S"], atol=g["coef_tol"])
    # stopping dates: 0 in the fixture means never exercised (our tau = m with zero payoff)
    h = np.maximum(K - S, 0.0)
    stop = [0 if h[t - 1, i] == 0 else t for i, t in enumerate(res["tau"])]
    assert stop == g["stopping_date_per_path"]


@pytest.mark.parametrize("seed", range(6))
def test_lsm_matches_independent_micro_oracle(seed):
    rng = np.random.default_rng(100 + seed)
    m, N, K, r, T = 3, 8, 1.0, 0.05, 1.0
    S = np.exp(rng.normal(0, 0.15, (m, N)).cumsum(axis=0)) * 0.97
    for tp in (oracle.PUT, oracle.CALL):
        a = oracle.lsm(S, tp, K, r, T, 2 if seed % 2 else 3, details=True)
        b = lsm_micro(S, tp, K, r, T, 2 if seed % 2 else 3)
        assert abs(a["price"] - b["price"]) < 1e-12
        np.testing.assert_array_equal(a["tau"], b["tau"])
        np.testing.assert_allclose(a["beta"], b["beta"], rtol=1e-6, atol=1e-9)  # normal equations square cond(X)
        assert a["degenerate_dates"] == b["degenerate_dates"]


def test_lsm_micro_oracle_on_sobol_paths():
    S = oracle.paths(36.0, .06, .2, 1.0, 6, 64, seed=1)
    a = oracle.lsm(S, oracle.PUT, 40.0, .06, 1.0, 3, details=True)
    b = lsm_micro(S, oracle.PUT, 40.0, .06, 1.0, 3)
    assert abs(a["price"] - b["price"]) < 1e-12
    np.testing.assert_array_equal(a["tau"], b["tau"])


def test_lsm_basis_choice_does_not_change_the_estimator():
    # {1, y, y^2} with y = S/K - 1 and {1, x, x^2} with x = S/K span the same
    # functions: same fitted values, same stopping dates, same price
    S = oracle.paths(100.0, .05, .3, 1.0, 12, 4096, seed=8)
    a = lsm_micro(S, oracle.PUT, 100.0, .05, 1.0, 3, center=1.0)
    b = lsm_micro(S, oracle.PUT, 100.0, .05, 1.0, 3, center=0.0)
    c = oracle.lsm(S, oracle.PUT, 100.0, .05, 1.0, 3, details=True)
    np.testing.assert_array_equal(a["tau"], b["tau"])
    np.testing.assert_array_equal(a["tau"], c["tau"])
    assert abs(a["price"] - b["price"]) < 1e-12 and abs(a["price"] - c["price"]) < 1e-12


def _rqmc(fn, R=16, base=1000):
    vals = np.array([fn(base + k) for k in range(R)])
    return vals.mean(), vals.std(ddof=1) / math.sqrt(R)


def test_european_limit_vs_black_scholes():
    for tp in (oracle.PUT, oracle.CALL):
        mean, se = _rqmc(lambda s: oracle.price(36, 40, .06, .2, 1.0, 16, 2 ** 12, type=tp, seed=s,
                                                rule=oracle.RULE_EUROPEAN)["price"])
        assert abs(mean - oracle.bs(tp, 36, 40, .06, .2, 1.0)) < 4 * se + 1e-4


def test_american_call_without_dividends_equals_european():
    mean, se = _rqmc(lambda s: oracle.price(100, 100, .05, .3, 1.0, 20, 2 ** 12, basis=3, type=oracle.CALL,
                                            seed=s)["price"])
    bs = oracle.bs(oracle.CALL, 100, 100, .05, .3, 1.0)
    assert abs(mean - bs) < 4 * se + 0.005 * bs


def test_american_at_least_european_and_intrinsic():
    for (S0, K) in [(36, 40), (44, 40), (30, 40)]:
        res = oracle.price(S0, K, .06, .2, 1.0, 50, 2 ** 13, basis=3, type=oracle.PUT, seed=1)
        eu = oracle.bs(oracle.PUT, S0, K, .06, .2, 1.0)
        assert res["price"] >= eu - 3 * res["std_err"]
        # t = 0 is not an exercise date, so the intrinsic bound is that of
        # exercising at t_1: E[e^{-r t_1}(K - S_1)^+] >= K e^{-r t_1} - S0 (Jensen)
        assert res["price"] >= max(K * math.exp(-.06 / 50) - S0, 0) - 3 * res["std_err"]


def test_lsm_vs_bermudan_crr_tree():
    m = 50
    mean, se = _rqmc(lambda s: oracle.price(36, 40, .06, .2, 1.0, m, 2 ** 13, basis=3, seed=s)["price"], R=8)
    tree = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, m, bermudan=True)
    assert abs(mean - tree) < 4 * se + 0.005 * tree


# ---------------------------------------------------------------- paper rule
def test_paper_rule_one_date_is_max_of_intrinsic_and_bs():
    for tp, S0 in [(oracle.PUT, 36.0), (oracle.CALL, 44.0), (oracle.PUT, 30.0)]:
        v = oracle.paper_ub_m1(tp, S0, 40.0, .06, .2, 1.0)
        assert v == max(max((40 - S0) if tp == oracle.PUT else (S0 - 40), 0.0), oracle.bs(tp, S0, 40, .06, .2, 1.0))


def test_paper_rule_is_discounted_pathwise_maximum():
    S0, K, r, sigma, T, m = 36.0, 40.0, .06, .2, 1.0, 7
    S = oracle.paths(S0, r, sigma, T, m, 512, seed=4)
    got = oracle.paper_ub(S, oracle.PUT, S0, K, r, sigma, T)["price"]
    dt = T / m
    full = np.vstack([np.full((1, 512), S0), S])           # dates 0..m
    h = np.maximum(K - full, 0.0)
    last = np.maximum(h[m - 1], [oracle.bs(oracle.PUT, s, K, r, sigma, dt) for s in full[m - 1]])
    terms = [np.exp(-r * j * dt) * h[j] for j in range(m - 1)] + [np.exp(-r * (m - 1) * dt) * last]
    assert abs(got - np.max(terms, axis=0).mean()) < 1e-12


def test_paper_rule_above_lsm_above_european():
    for tp, S0 in [(oracle.PUT, 36.0), (oracle.CALL, 44.0)]:
        S = oracle.paths(S0, .06, .2, 1.0, 25, 2 ** 12, seed=9)
        ub = oracle.paper_ub(S, tp, S0, 40.0, .06, .2, 1.0)["price"]
        ls = oracle.lsm(S, tp, 40.0, .06, 1.0, 3)["price"]
        eu = oracle.european(S, tp, 40.0, .06, 1.0)["price"]
        assert ub >= ls >= eu - 0.01


# ---------------------------------------------------------------- Greeks
def test_european_pathwise_greeks_vs_closed_form():
    S0, K, r, sigma, T = 100.0, 100.0, .05, .3, 1.0
    d1 = (math.log(S0 / K) + (r + .5 * sigma ** 2) * T) / (sigma * math.sqrt(T))
    g = [oracle.greeks(S0, K, r, sigma, T, 8, 2 ** 12, type=oracle.PUT, seed=s, rule=oracle.RULE_EUROPEAN)
         for s in range(8)]
    delta = np.mean([x["delta"] for x in g])
    vega = np.mean([x["vega"] for x in g])
    Nd1 = 0.5 * math.erfc(-d1 / math.sqrt(2))
    assert abs(delta - (Nd1 - 1)) < 2e-3
    assert abs(vega - S0 * math.exp(-.5 * d1 * d1) / math.sqrt(2 * math.pi) * math.sqrt(T)) < 0.2


def test_lsm_pathwise_greeks_vs_central_differences():
    # enough paths that exercise-boundary crossings under the bump average out
    S0, K, r, sigma, T, m, N = 36.0, 40.0, .06, .2, 1.0, 10, 2 ** 16
    g = oracle.greeks(S0, K, r, sigma, T, m, N, basis=3, seed=5)
    bS, bv = 1e-3 * S0, 1e-3 * sigma
    up = oracle.price(S0 + bS, K, r, sigma, T, m, N, basis=3, seed=5)["price"]
    dn = oracle.price(S0 - bS, K, r, sigma, T, m, N, basis=3, seed=5)["price"]
    vu = oracle.price(S0, K, r, sigma + bv, T, m, N, basis=3, seed=5)["price"]
    vd = oracle.price(S0, K, r, sigma - bv, T, m, N, basis=3, seed=5)["price"]
    fd_delta, fd_vega = (up - dn) / (2 * bS), (vu - vd) / (2 * bv)
    assert abs(g["delta"] - fd_delta) < 0.02 * abs(fd_delta) + 5e-3
    assert abs(g["vega"] - fd_vega) < 0.05 * abs(fd_vega) + 0.2
    base = oracle.price(S0, K, r, sigma, T, m, N, basis=3, seed=5)["price"]
    assert abs(g["price"] - base) < 1e-12


# ------------------------------------------------ boundary valuation (second pass)
def _fit(seed, m=50, n=2 ** 13, p=3):
    S = oracle.paths(36.0, .06, .2, 1.0, m, n, seed)
    return S, oracle.lsm(S, oracle.PUT, 40.0, .06, 1.0, p, details=True)


def test_boundary_valuation_on_fitting_paths_repeats_in_sample_decisions():
    S, fit = _fit(1)
    val = oracle.value_boundary(S, oracle.PUT, 40.0, .06, 1.0, fit["beta"], fit["deg"], details=True)
    assert val["price"] == fit["price"] and val["std_err"] == fit["std_err"]
    assert np.array_equal(val["tau"], fit["tau"])
    assert val["degenerate_dates"] == fit["degenerate_dates"]


def test_cash_flows_under_a_boundary_match_brute_force():
    """The per-date cash flows of the boundary valuation (what the
    regression of each date is fitted to under that boundary) against a
    pure-Python loop over paths and dates (oracle/micro.py), entry by entry,
    for a put and a call, with a degenerate date, an ITM-everywhere boundary
    and the fitted one."""
    from oracle.micro import cash_flows_under_boundary
    for tp, S0, K, seed in ((oracle.PUT, 36.0, 40.0, 5), (oracle.CALL, 44.0, 40.0, 6)):
        m, n, r, T = 7, 40, .06, 1.0
        S = oracle.paths(S0, r, .3, T, m, n, seed)
        fit = oracle.lsm(S, tp, K, r, T, 3, details=True)
        rng = np.random.default_rng(seed)
        for beta, deg in ((fit["beta"], fit["deg"]),
                          (rng.normal(0.0, 2.0, (m, 3)), (np.arange(m) == 3).astype(np.int32)),
                          (np.full((m, 2), -1e300), np.zeros(m, dtype=np.int32))):
            got = oracle.value_boundary(S, tp, K, r, T, beta, deg, cf_dates=True)["cf_dates"]
            ref = cash_flows_under_boundary(S, tp, K, r, T, beta, deg)
            np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14)


def test_regressions_on_the_cash_flows_under_the_fitted_boundary_reproduce_it():
    """Regressing each date's cash flows under the oracle's own fitted
    boundary (in-the-money paths, the oracle's normal equations) gives back
    the coefficients the LSM sweep fitted at that date: the cash flows are
    exactly the ones the sweep regressed on."""
    for tp, S0, p, seed in ((oracle.PUT, 36.0, 3, 7), (oracle.CALL, 44.0, 4, 8)):
        m, K, r, T = 30, 40.0, .06, 1.0
        S = oracle.paths(S0, r, .25, T, m, 4096, seed)
        fit = oracle.lsm(S, tp, K, r, T, p, details=True)
        cfd = oracle.value_boundary(S, tp, K, r, T, fit["beta"], fit["deg"], cf_dates=True)["cf_dates"]
        checked = 0
        for j in range(1, m):
            if fit["deg"][j - 1]:
                continue
            h = np.maximum(S[j - 1] - K, 0.0) if tp == oracle.CALL else np.maximum(K - S[j - 1], 0.0)
            I = h > 0
            y = S[j - 1][I] / K - 1.0
            X = np.vander(y, p, increasing=True)
            beta = oracle.solve_normal(X.T @ X, X.T @ cfd[j - 1][I])
            fitted, ref = X @ beta, X @ fit["beta"][j - 1]
            assert np.max(np.abs(fitted - ref)) <= 1e-9 * K, (j, np.max(np.abs(fitted - ref)))
            checked += 1
        assert checked >= m // 2


def test_boundary_without_exercise_is_the_european_estimator():
    S, fit = _fit(2)
    m = S.shape[0]
    val = oracle.value_boundary(S, oracle.PUT, 40.0, .06, 1.0, fit["beta"], np.ones(m, dtype=np.int32))
    eu = oracle.european(S, oracle.PUT, 40.0, .06, 1.0)
    assert val["price"] == pytest.approx(eu["price"], rel=1e-13)
    assert val["degenerate_dates"] == m - 1


def test_boundary_exercise_whenever_in_the_money_is_first_hitting_time():
    m, n, K, r, T = 12, 4096, 40.0, .06, 1.0
    S = oracle.paths(36.0, r, .2, T, m, n, 3)
    beta = np.zeros((m, 3))
    beta[:, 0] = -1e300                      # continuation below any positive payoff
    val = oracle.value_boundary(S, oracle.PUT, K, r, T, beta, np.zeros(m, dtype=np.int32), details=True)
    h = np.maximum(K - S, 0.0)               # [m, n]
    itm = h[:-1] > 0.0
    first = np.where(itm.any(axis=0), itm.argmax(axis=0) + 1, m)    # first in-the-money date, else maturity
    t = first * (T / m)
    ref = np.mean(h[first - 1, np.arange(n)] * np.exp(-r * t))
    assert np.array_equal(val["tau"], first)
    assert val["price"] == pytest.approx(ref, rel=1e-12)


def test_out_of_sample_price_is_low_biased_against_the_bermudan_tree():
    fit, val = oracle.price_oos(36.0, 40.0, .06, .2, 1.0, 50, 2 ** 14, basis=3, type=oracle.PUT, seed=1,
                                value_seed=2)
    tree = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, 50, bermudan=True)
    assert val["price"] <= tree + 3.0 * val["std_err"]
    assert val["price"] >= tree - 0.01 * tree
    assert val["price"] > oracle.bs(oracle.PUT, 36.0, 40.0, .06, .2, 1.0)


# ------------------------------------------- value vs number of exercise dates
def test_fig1_shape_in_the_oracle():
    """One date is the European estimator; the LSM value grows with nested
    date grids (within the RQMC error) toward the American tree value; the
    paper's pathwise rule stays above LSM."""
    import workloads
    dates = (1, 2, 4, 8, 16, 32, 64)
    lsm = {o.n_steps: oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, 2 ** 13, basis=o.basis, seed=o.seed)
           for o in workloads.fig1_options(dates, rules=(oracle.RULE_LSM,))}
    ub = {o.n_steps: oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, 2 ** 13, seed=o.seed, rule=o.rule)
          for o in workloads.fig1_options(dates, rules=(oracle.RULE_PAPER_UB,))}
    S1 = oracle.paths(36.0, .06, .2, 1.0, 1, 2 ** 13, 21)
    assert lsm[1]["price"] == pytest.approx(oracle.european(S1, oracle.PUT, 40.0, .06, 1.0)["price"], rel=1e-14)
    for a, b in zip(dates, dates[1:]):
        assert lsm[b]["price"] >= lsm[a]["price"] - 3 * (lsm[a]["std_err"] + lsm[b]["std_err"])
    american = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000)
    assert american - 0.03 * american <= lsm[64]["price"] <= american + 3 * lsm[64]["std_err"]
    assert lsm[64]["price"] - lsm[1]["price"] > 0.5          # early exercise is worth ~0.6 here
    for m in dates:
        assert ub[m]["price"] >= lsm[m]["price"] - 3 * lsm[m]["std_err"]


# ------------------------------------------ the paper's LCG-permuted points
@pytest.mark.parametrize("N", [1, 2, 3, 1000, 4096, 12345])
def test_lcg_permutation_is_a_bijection(N):
    for d in (0, 5):
        p = oracle.lcg_perm(11, d, N, np.arange(N))
        assert np.array_equal(np.sort(p), np.arange(N))


def test_lcg_map_has_full_period():
    """Hull-Dobell: a = 1 mod 4, c odd => x -> a x + c (mod 2^k) is one cycle."""
    a, c, M = oracle.lcg_params(3, 4, 1000)
    assert M == 1024
    for d in range(4):
        assert a[d] % 4 == 1 and c[d] % 2 == 1
        x, seen = 0, set()
        for _ in range(M):
            seen.add(x)
            x = (int(a[d]) * x + int(c[d])) % M
        assert x == 0 and len(seen) == M


def test_permuted_paths_rebuilt_from_scipy_points():
    """Path i = GBM of the bridge of ndtri(u) of the unshifted Sobol' points
    pi_d(i) (scipy's points, the pinned bridge matrix)."""
    from scipy.stats import qmc
    from scipy.special import ndtri
    m, N, seed, S0, r, sig, T = 16, 700, 9, 36.0, .06, .2, 1.0
    S = oracle.paths_permuted(S0, r, sig, T, m, N, seed)
    pts = qmc.Sobol(d=m, scramble=False, bits=32).random(1024)
    X = np.round(pts * 2.0 ** 32).astype(np.uint64)            # integer points 0..1023
    A = oracle.bridge_matrix(m, T)
    t = np.arange(1, m + 1) * (T / m)
    for i in (0, 1, 2, 345, 699):
        j = [int(oracle.lcg_perm(seed, d, N, i)[0]) for d in range(m)]
        u = (X[j, np.arange(m)].astype(np.float64) + 0.5) / 2.0 ** 32
        W = A @ ndtri(u)
        want = S0 * np.exp((r - 0.5 * sig * sig) * t + sig * W)
        np.testing.assert_allclose(S[:, i], want, rtol=1e-12)


def test_permuted_points_give_an_unbiased_lsm_price():
    p_perm = [oracle.lsm(oracle.paths_permuted(36., .06, .2, 1., 16, 2 ** 12, s), oracle.PUT, 40., .06, 1., 3)
              for s in range(6)]
    mean = np.mean([q["price"] for q in p_perm])
    se = np.std([q["price"] for q in p_perm], ddof=1) / np.sqrt(len(p_perm))
    ref = oracle.price(36., 40., .06, .2, 1., 16, 2 ** 16, basis=3, seed=1)
    assert abs(mean - ref["price"]) < 4 * se + 3 * ref["std_err"] + 0.01



# ------------------------------------------------ dual upper bound (primal-dual)
def test_dual_normals_are_counter_based_splitmix64():
    """Inner path k from date j of outer path i owns ceil(m/2) consecutive
    SplitMix64 outputs; steps 2q-1 and 2q take the high and low halves of
    the q-th (recomputed here from SplitMix64's published constants)."""
    from scipy.special import ndtri
    M64 = (1 << 64) - 1

    def sm64_at(seed, n):
        z = (seed + n * 0x9E3779B97F4A7C15) & M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    m, n_in = 7, 5
    H = (m + 1) // 2
    for (i, j, k, s) in [(0, 1, 0, 1), (0, 1, 0, 2), (3, 2, 4, 5), (3, 2, 4, 6), (11, 6, 2, 1)]:
        out = sm64_at(9, ((i * m + j - 1) * n_in + k) * H + (s + 1) // 2)
        x = out >> 32 if s % 2 else out & 0xFFFFFFFF
        assert oracle.dual_normal(9, m, n_in, i, j, k, s) == pytest.approx(ndtri((x + 0.5) / 2.0 ** 32), rel=1e-13)
    # consecutive inner paths own disjoint outputs: the last step of path k and the first of path k+1 differ
    assert oracle.dual_normal(9, m, n_in, 0, 1, 0, m - 1) != oracle.dual_normal(9, m, n_in, 0, 1, 1, 1)


def test_dual_with_one_date_is_the_european_estimator():
    S = oracle.paths(36.0, .06, .2, 1.0, 1, 3000, 4)
    d = oracle.dual_upper(S, oracle.PUT, 40.0, .06, .2, 1.0, np.zeros((1, 3)), np.ones(1, dtype=np.int32), 8, 1,
                          details=True)
    eu = oracle.european(S, oracle.PUT, 40.0, .06, 1.0)["price"]
    assert d["L0"] == pytest.approx(eu, rel=1e-13)
    np.testing.assert_allclose(d["U"], eu, rtol=1e-13)


def test_dual_matches_a_brute_force_loop():
    """Pure-Python restatement on a tiny case: inner paths, L, M, max."""
    import math
    m, N, n_in, K, r, sig, T, seed_in = 3, 5, 3, 40.0, .06, .2, 1.0, 7
    S = oracle.paths(36.0, r, sig, T, m, N, 3)
    fit = oracle.lsm(oracle.paths(36.0, r, sig, T, m, 64, 1), oracle.PUT, K, r, T, 2, details=True)
    beta, deg = fit["beta"], fit["deg"]
    dt = T / m
    h = lambda x: max(K - x, 0.0)

    def stops(j, x):
        if j >= m:
            return True
        if deg[j - 1] or not h(x) > 0:
            return False
        y = x / K - 1
        return h(x) > sum(beta[j - 1][q] * y ** q for q in range(beta.shape[1]))

    Q = np.zeros((N, m))
    for i in range(N):
        for j in range(1, m):
            tot = 0.0
            for k in range(n_in):
                x, v = S[j - 1, i], 0.0
                for s in range(1, m - j + 1):
                    z = oracle.dual_normal(seed_in, m, n_in, i, j, k, s)
                    x = x * math.exp((r - sig * sig / 2) * dt + sig * math.sqrt(dt) * z)
                    if stops(j + s, x):
                        v = math.exp(-r * s * dt) * h(x)
                        break
                tot += v
            Q[i, j] = tot / n_in
    L1 = [math.exp(-r * dt) * (h(S[0, i]) if stops(1, S[0, i]) else Q[i, 1]) for i in range(N)]
    L0 = sum(L1) / N
    U = []
    for i in range(N):
        Mj, prev, best = 0.0, L0, -1e300
        for j in range(1, m + 1):
            D = math.exp(-r * j * dt)
            Z = D * h(S[j - 1, i])
            if j == m:
                L, DQ = Z, 0.0
            else:
                DQ = D * Q[i, j]
                L = Z if stops(j, S[j - 1, i]) else DQ
            Mj += L - prev
            prev = DQ
            best = max(best, Z - Mj)
        U.append(best)
    d = oracle.dual_upper(S, oracle.PUT, K, r, sig, T, beta, deg, n_in, seed_in, details=True)
    assert d["L0"] == pytest.approx(L0, rel=1e-12)
    np.testing.assert_allclose(d["U"], U, rtol=1e-12)


def test_dual_and_lower_bound_bracket_the_bermudan_tree():
    m = 10
    fit, low, up = oracle.price_dual(36.0, 40.0, .06, .2, 1.0, m, 2 ** 13, 1024, 128, basis=3, seed=1, outer_seed=2,
                                     seed_in=3)
    tree = oracle.crr(oracle.PUT, 36, 40, .06, .2, 1.0, 10000, m, bermudan=True)
    assert low["price"] <= tree + 3 * low["std_err"]
    assert up["upper"] >= tree - 3 * up["std_err"]
    assert up["upper"] - low["price"] < 0.03 * tree
    # far below the perfect-foresight bound E[max_j Z_j] on the same outer paths
    S = oracle.paths(36.0, .06, .2, 1.0, m, 1024, 2)
    disc = np.exp(-.06 * np.arange(1, m + 1)[:, None] / m)
    foresight = np.mean(np.max(disc * np.maximum(40.0 - S, 0.0), axis=0))
    assert up["upper"] < foresight - 0.1


def test_oracle_results_do_not_depend_on_its_thread_count():
    """OpenMP runs only across independent paths; sums are taken in a fixed
    order, so one thread and all threads give the same bits."""
    n0 = oracle.threads()
    S = oracle.paths(36.0, .06, .2, 1.0, 12, 3001, 5)
    fit = oracle.lsm(S, oracle.PUT, 40.0, .06, 1.0, 3, details=True)
    d = oracle.dual_upper(S[:, :40], oracle.PUT, 40.0, .06, .2, 1.0, fit["beta"], fit["deg"], 16, 3)
    try:
        oracle.set_threads(1)
        assert oracle.threads() == 1
        S1 = oracle.paths(36.0, .06, .2, 1.0, 12, 3001, 5)
        fit1 = oracle.lsm(S1, oracle.PUT, 40.0, .06, 1.0, 3, details=True)
        d1 = oracle.dual_upper(S1[:, :40], oracle.PUT, 40.0, .06, .2, 1.0, fit1["beta"], fit1["deg"], 16, 3)
    finally:
        oracle.set_threads(n0)
    assert oracle.threads() == n0
    assert np.array_equal(S, S1)
    assert fit["price"] == fit1["price"] and np.array_equal(fit["beta"], fit1["beta"])
    assert d == d1


def test_standard_errors_are_the_sample_deviation_of_the_discounted_path_values():
    """Every estimator's std_err is the sample standard deviation (N - 1) of
    the per-path values discounted to t = 0, over sqrt(N), and its price is
    their mean (Eqs. 6-8): recomputed in numpy from the paths, the stopping
    dates and the per-path values, for LSM, its out-of-sample valuation, the
    European estimator, the paper's rule and the dual bound."""
    S0, K, r, sigma, T, m, N = 36.0, 40.0, .06, .2, 1.0, 9, 3000
    dt = T / m
    S = oracle.paths(S0, r, sigma, T, m, N, seed=9)
    idx = np.arange(N)

    def check(res, v, key="price"):
        assert abs(res[key] - v.mean()) < 1e-12 * max(1.0, abs(v.mean()))
        assert abs(res["std_err"] - v.std(ddof=1) / math.sqrt(N)) < 1e-12 * v.std()

    fit = oracle.lsm(S, oracle.PUT, K, r, T, 3, details=True)
    tau = fit["tau"].astype(np.int64)
    assert tau.min() >= 1 and tau.max() <= m
    check(fit, np.exp(-r * tau * dt) * np.maximum(K - S[tau - 1, idx], 0.0))

    S2 = oracle.paths(S0, r, sigma, T, m, N, seed=10)
    val = oracle.value_boundary(S2, oracle.PUT, K, r, T, fit["beta"], fit["deg"], details=True)
    t2 = val["tau"].astype(np.int64)
    check(val, np.exp(-r * t2 * dt) * np.maximum(K - S2[t2 - 1, idx], 0.0))

    check(oracle.european(S, oracle.CALL, K, r, T), np.exp(-r * T) * np.maximum(S[-1] - K, 0.0))

    full = np.vstack([np.full((1, N), S0), S])
    h = np.maximum(K - full, 0.0)
    last = np.maximum(h[m - 1], [oracle.bs(oracle.PUT, s, K, r, sigma, dt) for s in full[m - 1]])
    V = np.max([np.exp(-r * j * dt) * h[j] for j in range(m - 1)] + [np.exp(-r * (m - 1) * dt) * last], axis=0)
    check(oracle.paper_ub(S, oracle.PUT, S0, K, r, sigma, T), V)

    So = oracle.paths(S0, r, sigma, T, m, 200, seed=11)
    up = oracle.dual_upper(So, oracle.PUT, K, r, sigma, T, fit["beta"], fit["deg"], 8, 5, details=True)
    U = up["U"]
    assert abs(up["upper"] - U.mean()) < 1e-12 * U.mean()
    assert abs(up["std_err"] - U.std(ddof=1) / math.sqrt(len(U))) < 1e-12 * U.std()


def test_too_few_in_the_money_paths_make_a_degenerate_date():
    """Reading of the degenerate-date rule: fewer than p paths strictly in
    the money at a date (a path at the strike is not) means no regression
    and no exercise there, counted once; with p at most that count the date
    is regressed.  Hand-made put paths, K = 1, 3 dates, 7 paths."""
    K, r, T = 1.0, 0.05, 3.0
    S = np.array([[0.50, 0.60, 0.70, 0.80, 1.20, 1.30, 1.40],     # date 1: 4 in the money
                  [0.10, 0.20, 1.00, 1.10, 1.20, 1.30, 1.40],     # date 2: 2 in the money (1.00 is at the strike)
                  [0.90, 0.95, 1.10, 0.97, 1.20, 0.99, 1.40]])    # maturity
    deep = oracle.lsm(S, oracle.PUT, K, r, T, 3, details=True)
    assert deep["n_itm"].tolist()[:2] == [4, 2]
    assert deep["deg"].tolist()[1] == 1 and deep["degenerate_dates"] == 1
    assert 2 not in deep["tau"].tolist()                           # deep in the money at date 2, yet never exercised
    two = oracle.lsm(S, oracle.PUT, K, r, T, 2, details=True)
    assert two["deg"].tolist()[1] == 0 and two["degenerate_dates"] == 0
    assert two["tau"].tolist()[:2] == [2, 2]                        # exact fit through the 2 points: exercise


def test_exercise_and_moneyness_tests_are_strict():
    """Reading of the tie-breaks: a path exercises only where its payoff
    strictly exceeds the continuation value, and only strictly in the money.
    A constant boundary (p = 1) of 0.25 K at date 1 and exact binary values:
    payoff 0.25 equals it (kept), 0.5 exceeds it (exercised); a path at the
    strike with a boundary below zero is not in the money (kept)."""
    K, r, T = 1.0, 0.0, 2.0
    S = np.array([[0.75, 0.50, 1.00],
                  [1.50, 1.50, 1.50]])                               # maturity: out of the money
    beta = np.array([[0.25], [0.0]])
    deg = np.array([0, 1], dtype=np.int32)
    res = oracle.value_boundary(S, oracle.PUT, K, r, T, beta, deg, details=True)
    assert res["tau"].tolist() == [2, 1, 2]
    assert res["price"] == 0.5 / 3
    below = oracle.value_boundary(S, oracle.PUT, K, r, T, np.array([[-1.0], [0.0]]), deg, details=True)
    assert below["tau"].tolist() == [1, 1, 2]                        # S = K is not exercised even against c < 0


@pytest.mark.parametrize("m", [13, 16])
def test_shifted_paths_rebuilt_from_scipy_points(m):
    """Steps 1-3 end to end: path i is the GBM (Eq. 9 in log space) of the
    bridge of ndtri((x + 1/2) 2^-32) of scipy's Sobol' point i (point 0
    included) XOR the digital shift of each dimension; a block starting at
    `first` is the same columns of the whole array."""
    from scipy.stats import qmc
    from scipy.special import ndtri
    N, seed, S0, r, sig, T = 600, 12, 100.0, .05, .3, 1.5
    S, W = oracle.paths(S0, r, sig, T, m, N, seed, with_W=True)
    pts = qmc.Sobol(d=m, scramble=False, bits=32).random(1024)
    X = np.round(pts * 2.0 ** 32).astype(np.uint64) ^ oracle.shifts(seed, m).astype(np.uint64)[None, :]
    A = oracle.bridge_matrix(m, T)
    t = np.arange(1, m + 1) * (T / m)
    for i in (0, 1, 2, 511, 599):
        u = (X[i].astype(np.float64) + 0.5) / 2.0 ** 32
        Wi = A @ ndtri(u)
        np.testing.assert_allclose(W[:, i], Wi, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(S[:, i], S0 * np.exp((r - 0.5 * sig * sig) * t + sig * Wi), rtol=1e-12)
    part = oracle.paths(S0, r, sig, T, m, 100, seed, first=450)
    np.testing.assert_array_equal(part, S[:, 450:550])
