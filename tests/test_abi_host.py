"""C-ABI library on the CPU: it loads, exports every function include/amc.h
declares, and its host-side logic (direction numbers, digital shifts, bridge
schedule, validation, launch plan) is right.  No compute call needs a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


def _declared():
    with open(os.path.join(ROOT, "include", "amc.h")) as f:
        src = f.read()
    # function declarations: a return type at the start of a line, then the name
    return sorted(set(re.findall(r"^(?:const\s+)?[a-z_0-9]+\s*\*?\s*(amc_[a-z_0-9]+)\s*\(", src, re.M)))


def test_exports_every_declared_function(amc):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(amc.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(amc.SIGNATURES), set(names) - set(amc.SIGNATURES)


def test_strerror_and_version(amc):
    assert amc.strerror(0) == "ok"
    assert "timed out" in amc.strerror(amc.AMC_ETIMEOUT)
    assert "cancel" in amc.strerror(amc.AMC_ECANCELED)
    assert amc.amc_version() >= 1


@pytest.mark.parametrize("m", [1, 2, 50, 252, 512])
def test_library_direction_numbers_reproduce_scipy_sobol(amc, m):
    from scipy.stats import qmc
    V = amc.amc_sobol_directions(m).astype(np.uint64)
    n = 256
    ref = np.round(qmc.Sobol(d=m, scramble=False, bits=32).random(n) * 2.0 ** 32).astype(np.uint64).T
    i = np.arange(n, dtype=np.uint64)
    g = i ^ (i >> 1)
    X = np.zeros((m, n), dtype=np.uint64)
    for b in range(32):
        X ^= np.where(((g >> b) & 1)[None, :] == 1, V[:, b:b + 1], 0)
    np.testing.assert_array_equal(X, ref)


def test_library_shifts_are_splitmix64_high_words(amc):
    import json
    with open(os.path.join(ROOT, "tests", "golden", "splitmix64_seed0.json")) as f:
        g = json.load(f)
    sh = amc.amc_digital_shifts(0, 3)
    assert [int(s) for s in sh] == [int(h, 16) >> 32 for h in g["outputs_hex"]]


@pytest.mark.parametrize("m", [1, 2, 3, 7, 16, 50, 252, 365, 512])
def test_library_bridge_schedule(amc, m):
    d, l, r = amc.amc_bridge_schedule(m)
    assert sorted(d.tolist()) == list(range(1, m + 1)) and d[0] == m
    seen = {0, m}
    for k in range(1, m):
        assert l[k] in seen and r[k] in seen and l[k] < d[k] < r[k] and d[k] == (l[k] + r[k]) // 2
        seen.add(int(d[k]))
    if m == 16:
        assert d.tolist() == [16, 8, 4, 12, 2, 6, 10, 14, 1, 3, 5, 7, 9, 11, 13, 15]


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 16, 50, 252, 365, 512])
def test_bridge_plan_evaluates_the_bridge_matrix(amc, m):
    """The depth-first plan the path-generation kernels run, evaluated here
    with its slot stack in FP64, gives W = A z with the oracle's bridge matrix
    A (pinned to A A^T = min(t_i, t_j)).  The stack starts at a finite value
    other than 0 as well: the result does not change, so every read of a slot
    not yet written in the pass (W(0) has no slot) carries weight 0."""
    import oracle
    p = amc.amc_bridge_plan(m)
    assert sorted(p["date"].tolist()) == list(range(1, m + 1)) and p["date"][0] == m
    assert sorted(p["coord"].tolist()) == list(range(m))
    assert 1 <= p["n_slots"] <= 11 and p["so"].max() < p["n_slots"]
    T = 1.3
    A = oracle.bridge_matrix(m, T)
    Z = np.random.default_rng(m).standard_normal((m, 3))
    for start in (0.0, 7.25):
        st = np.full((p["n_slots"], 3), start)
        W = np.zeros((m, 3))
        for k in range(m):
            w = p["wl"][k] * st[p["sl"][k]] + p["wr"][k] * st[p["sr"][k]] + p["sdu"][k] * np.sqrt(T / m) * Z[p["coord"][k]]
            st[p["so"][k]] = w
            W[p["date"][k] - 1] = w
        np.testing.assert_allclose(W, A @ Z, rtol=1e-12, atol=1e-12)


def test_bridge_plan_rejects_bad_sizes(amc):
    for m in (0, -1, amc.AMC_MAX_STEPS + 1):
        with pytest.raises(amc.AmcError) as ei:
            amc.amc_bridge_plan(m)
        assert ei.value.code == amc.AMC_EINVAL


def test_validation(amc):
    import workloads
    good = workloads.single_small()
    assert amc.amc_validate_option(good) == 0
    inf, nan = float("inf"), float("nan")
    for field, bad in [("S0", 0.0), ("S0", -36.0), ("S0", inf), ("S0", nan), ("K", -1.0), ("K", 0.0), ("K", inf),
                       ("sigma", nan), ("sigma", 0.0), ("sigma", -0.2), ("sigma", inf), ("T", 0.0), ("T", -1.0),
                       ("T", inf), ("r", inf), ("r", -inf), ("r", nan), ("n_steps", 0), ("n_steps", -1),
                       ("n_steps", 513), ("n_paths", 0), ("n_paths", -5), ("n_paths", 2 ** 31 + 1), ("basis", 0),
                       ("basis", 5), ("type", 2), ("type", -1), ("rule", 3), ("rule", -1)]:
        d = good.as_dict()
        d[field] = bad
        assert amc.amc_validate_option(d) == amc.AMC_EINVAL, (field, bad)
    # the limits themselves are valid, as are a negative rate and, outside LSM, any basis
    for field, ok in [("n_steps", 1), ("n_steps", 512), ("n_paths", 1), ("n_paths", 2 ** 31), ("basis", 1),
                      ("basis", 4), ("r", -0.02), ("r", 0.0)]:
        d = good.as_dict()
        d[field] = ok
        assert amc.amc_validate_option(d) == 0, (field, ok)
    for rule in (amc.AMC_RULE_PAPER_UB, amc.AMC_RULE_EUROPEAN):
        d = dict(good.as_dict(), rule=rule, basis=0)
        assert amc.amc_validate_option(d) == 0, rule


def test_path_layout(amc):
    assert amc.amc_path_ld(1) == 32 and amc.amc_path_ld(32) == 32 and amc.amc_path_ld(33) == 64
    assert amc.amc_path_bytes(252, 2 ** 20, amc.AMC_MIXED) == 252 * 2 ** 20 * 4
    assert amc.amc_path_bytes(50, 1000, amc.AMC_FP64) == 50 * 1024 * 8


def test_sweep_plan_is_a_function_of_paths(amc):
    for n in [1, 1000, 2 ** 14, 2 ** 18, 2 ** 20, 2 ** 20 + 7]:
        ctas, ppt = amc.amc_plan_sweep(n, 152, amc.AMC_FP64, amc.AMC_RULE_LSM)
        assert ctas * 256 * ppt >= n
        assert ctas * 256 * ppt < n + 256 * ppt + 1
        assert ppt in (4, 8, 16, 32)
        ctas, ppt = amc.amc_plan_sweep(n, 152, amc.AMC_MIXED, amc.AMC_RULE_LSM)
        if n <= 2 ** 18:        # one cluster of up to 16 CTAs of 16384 paths
            assert ppt == 16 and ctas == -(-n // 16384) and ctas <= 16
        else:                   # CTAs of 7680 paths exchanging through L2
            assert ppt == 8 and ctas == -(-n // 7680) and ctas <= 152
    assert amc.amc_plan_sweep(2 ** 18, 152, amc.AMC_MIXED, amc.AMC_RULE_LSM) == (16, 16)
    assert amc.amc_plan_sweep(2 ** 18 + 1, 152, amc.AMC_MIXED, amc.AMC_RULE_LSM) == (35, 8)
    assert amc.amc_plan_sweep(2 ** 20, 152, amc.AMC_FP64, amc.AMC_RULE_LSM) == (512, 8)
    assert amc.amc_plan_sweep(2 ** 20, 152, amc.AMC_MIXED, amc.AMC_RULE_LSM) == (137, 8)
    assert amc.amc_plan_sweep(2 ** 20, 152, amc.AMC_MIXED, amc.AMC_RULE_EUROPEAN) == (512, 8)
    for prec in (amc.AMC_FP64, amc.AMC_MIXED):
        with pytest.raises(amc.AmcError):
            amc.amc_plan_sweep(2 ** 31, 152, prec, amc.AMC_RULE_LSM)


@pytest.mark.parametrize("n", [1, 3, 1000, 12345, 2 ** 20])
def test_library_lcg_permutation_parameters(amc, n):
    """The library's LCG parameters (its own SplitMix64 stream) equal the
    definition: a = 1 mod 4, c odd, M the least power of two >= n."""
    import oracle
    a, c, M = amc.amc_lcg_params(77, 40, n)
    ao, co, Mo = oracle.lcg_params(77, 40, n)
    assert M == Mo and M >= n and (M == 1 or M < 2 * n)
    np.testing.assert_array_equal(a.astype(np.uint64), ao)
    np.testing.assert_array_equal(c.astype(np.uint64), co)
    if M >= 4:
        assert np.all(a % 4 == 1) and np.all(c % 2 == 1)


def test_host_helpers_reject_bad_arguments(amc):
    """Every host-only helper returns AMC_EINVAL for arguments outside its
    documented range, and the size helpers return 0 for empty inputs."""
    def einval(fn, *args):
        with pytest.raises(amc.AmcError) as ei:
            fn(*args)
        assert ei.value.code == amc.AMC_EINVAL, (fn.__name__, args)

    for m in (0, amc.AMC_MAX_STEPS + 1):
        einval(amc.amc_sobol_directions, m)
        einval(amc.amc_bridge_schedule, m)
    assert amc.amc_sobol_directions(amc.AMC_MAX_STEPS).shape == (amc.AMC_MAX_STEPS, 32)
    assert sorted(amc.amc_bridge_schedule(amc.AMC_MAX_STEPS)[0].tolist()) == list(range(1, amc.AMC_MAX_STEPS + 1))
    assert amc.lib().amc_digital_shifts(1, -1, None) == amc.AMC_EINVAL      # below the binding's numpy sizing
    assert amc.amc_digital_shifts(1, 0).shape == (0,)
    for n_dims, n_points in ((0, 10), (amc.AMC_MAX_STEPS + 1, 10), (3, 0), (3, 2 ** 31 + 1)):
        einval(amc.amc_lcg_params, 5, n_dims, n_points)
    for n_paths, sms in ((0, 152), (-1, 152), (1000, 0)):
        einval(amc.amc_plan_sweep, n_paths, sms)
    assert amc.amc_path_ld(0) == 0 and amc.amc_path_ld(-3) == 0
    assert amc.amc_path_bytes(0, 100, amc.AMC_MIXED) == 0 and amc.amc_path_bytes(10, 0, amc.AMC_FP64) == 0
    for code in (amc.AMC_EINVAL, amc.AMC_ENOMEM, amc.AMC_ECUDA, amc.AMC_EBUSY, amc.AMC_PENDING, amc.AMC_ENOTFOUND):
        assert amc.strerror(code) and amc.strerror(code) != amc.strerror(0)
    assert amc.strerror(-12345)                                     # unknown codes still get a string
