"""The replay check of a mixed-precision LSM sweep (tests/lsm_replay.py),
tested on the CPU against a numpy FP32 sweep that follows the kernel's
arithmetic: y = fma(S, fl(1/K), -1) in FP32, FP32 cash flows discounted by
fl(e^{-r dt}) once per date, FP32 sums over 8 paths per thread and then a
pairwise tree, an FP64 solve of the oracle's equilibrated normal equations,
FP32 coefficients and a Horner evaluation by FMAs in FP32.

On the options where the LSM estimator is unstable at FP32 precision (the
ones whose mixed price cannot match the FP64 oracle's within 2e-4 K), this
faithful FP32 sweep must pass the check; the same sweep with a planted
mistake (a dropped moment term, a wrong discount, a reversed exercise test,
a wrong right-hand side index) must fail it.  So the check's bounds are
neither too tight for FP32 arithmetic nor loose enough to let a kernel bug
through.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from lsm_replay import replay_check

f32 = np.float32


def _fma32(a, b, c):
    # a*b of two FP32 numbers is exact in FP64; one rounding to FP32
    return (a.astype(np.float64) * b.astype(np.float64) + np.asarray(c, np.float64)).astype(f32)


def _sum32(v):
    """FP32 sum: 8 terms per thread in order, then a pairwise tree."""
    v = np.concatenate([v.astype(f32), np.zeros((-len(v)) % 8, f32)]).reshape(-1, 8)
    acc = np.zeros(v.shape[0], f32)
    for k in range(8):
        acc = (acc + v[:, k]).astype(f32)
    while len(acc) > 1:
        acc = np.concatenate([acc, np.zeros(len(acc) % 2, f32)])
        acc = (acc[0::2] + acc[1::2]).astype(f32)
    return float(acc[0]) if len(acc) else 0.0


def fp32_sweep(S32, o, plant=None):
    """FP32 LSM sweep on FP32 paths S32 [m, N]; returns (coef [m, 5] in units
    of K on the y basis, result dict).  `plant` names a mistake to plant."""
    m, N = S32.shape
    p, put = o.basis, o.type == oracle.PUT
    invK = f32(1.0 / o.K)
    disc = f32(math.exp(-o.r * o.T / m))
    if plant == "discount":
        disc = f32(math.exp(-o.r * o.T / m * 1.01))
    y = _fma32(S32.astype(f32), np.full_like(S32, invK, dtype=f32), -1.0)
    itm = (y < 0) if put else (y > 0)
    h = np.where(itm, -y if put else y, f32(0))
    coef = np.zeros((m, 5))
    coef[m - 1, 4] = 1.0
    cf = h[m - 1].copy()
    degenerate = 0
    for j in range(m - 1, 0, -1):
        row = j - 1
        cf = (cf * disc).astype(f32)
        I = itm[row]
        yI = y[row][I]
        yy = (yI * yI).astype(f32)
        y3 = (yy * yI).astype(f32)
        terms = [np.ones_like(yI), yI, yy, y3, (yy * yy).astype(f32), (yy * y3).astype(f32), (y3 * y3).astype(f32)]
        if plant == "moment":
            terms[3] = (yy * yy).astype(f32)
        M = [_sum32(terms[q]) for q in range(2 * p - 1)]
        cI = cf[I]
        rk = [0, 1, 2, 3] if plant != "rhs_index" else [0, 2, 1, 3]
        R = np.array([_sum32((cI * terms[rk[k]]).astype(f32)) for k in range(p)])
        G = np.array([[M[k + l] for l in range(p)] for k in range(p)])
        beta = None if int(I.sum()) < p else oracle.solve_normal(G, R)
        if beta is None:
            degenerate += 1
            coef[row, 4] = 1.0
            continue
        b = beta.astype(f32)
        coef[row, :p] = b
        cont = np.full_like(yI, b[p - 1])
        for k in range(p - 2, -1, -1):
            cont = _fma32(cont, yI, b[k])
        hI = h[row][I]
        ex = (hI < cont) if plant == "exercise" else (hI > cont)
        cI = cI.copy()
        cI[ex] = hI[ex]
        cf[I] = cI
    price = math.exp(-o.r * o.T / m) * o.K * float(np.mean(cf.astype(np.float64)))
    return coef, {"price": price, "status": 0, "degenerate_dates": degenerate}


UNSTABLE = {
    "huge_vol": workloads.Option(100.0, 100.0, 0.05, 1.5, 1.0, 50, 8192, basis=4, seed=21),
    "long_call": workloads.Option(50.0, 60.0, 0.08, 0.4, 10.0, 120, 8192, basis=4, type=1, seed=26),
    "ls_table1": workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 8192, basis=3, seed=1),
}


def _fp32_paths(o):
    return oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed).astype(f32).astype(np.float64)


@pytest.mark.parametrize("name", sorted(UNSTABLE))
def test_faithful_fp32_sweep_passes_the_replay_check(name):
    o = UNSTABLE[name]
    S = _fp32_paths(o)
    coef, res = fp32_sweep(S, o)
    d = replay_check(S, o, coef, res)
    assert d["residual_ratio"] <= 1.0 and d["price_ratio"] <= 1.0, d


@pytest.mark.parametrize("plant", ["moment", "discount", "exercise", "rhs_index"])
def test_planted_sweep_mistakes_fail_the_replay_check(plant):
    o = UNSTABLE["huge_vol"]
    S = _fp32_paths(o)
    coef, res = fp32_sweep(S, o, plant=plant)
    with pytest.raises(AssertionError):
        replay_check(S, o, coef, res)


def test_unstable_cases_really_miss_the_oracle_in_fp32():
    """Why the check exists: on these options the faithful FP32 sweep's
    price is more than 2e-4 K away from the FP64 oracle's on the same
    (FP32) paths, although every date passes the replay check."""
    missed = 0
    for name in ("huge_vol", "long_call"):
        o = UNSTABLE[name]
        S = _fp32_paths(o)
        _, res = fp32_sweep(S, o)
        ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"]
        missed += abs(res["price"] - ref) > 2e-4 * o.K
    assert missed >= 1
