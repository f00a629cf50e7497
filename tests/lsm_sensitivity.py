"""Sensitivity of the LSM estimator to FP32 arithmetic, measured with the
oracle (test helper, CPU): its price under path noise at the FP32 paths'
error level, and under FP32 sums in the sweep's order.  Written in numpy
from the sweep's definition (oracle paths and solve)."""
import numpy as np

import oracle


def paths(o):
    return oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed)


def path_noise_spread(o, eps=2e-5, reps=4):
    S = paths(o)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"]
    return max(abs(oracle.lsm(S * (1 + eps * np.random.default_rng(k).standard_normal(S.shape)), o.type, o.K, o.r,
                              o.T, o.basis)["price"] - ref) / o.K for k in range(reps))


def fp32_noise_spread(o):
    """The oracle price's largest move under relative path noise at the FP32
    paths' error level: 4 draws at 2e-5 (their largest deviation) and 4 at
    1e-6 (their typical one).  Two draws at one level missed an unstable
    served call (LSM below the European value) by a factor of three."""
    return max(path_noise_spread(o, eps=2e-5, reps=4), path_noise_spread(o, eps=1e-6, reps=4))


def lsm_fp32_sums(S, o):
    """LSM (units of K, moneyness basis) with FP32 cash flows and FP32
    per-thread (8 paths) + pairwise sums of the moments and right-hand
    sides, the FP64 solve of the oracle."""
    m, N = S.shape
    p, put = o.basis, o.type == oracle.PUT
    disc = np.float32(np.exp(-o.r * o.T / m))
    y_all = (S / o.K - 1.0).astype(np.float32)
    h_all = np.maximum(-y_all if put else y_all, np.float32(0))
    cf = h_all[m - 1].copy()

    def fsum(v):
        v = np.concatenate([v.astype(np.float32), np.zeros((-len(v)) % 8, np.float32)]).reshape(-1, 8)
        acc = np.zeros(v.shape[0], np.float32)
        for k in range(8):
            acc = acc + v[:, k]
        while len(acc) > 1:
            acc = np.concatenate([acc, np.zeros(len(acc) % 2, np.float32)])
            acc = acc[0::2] + acc[1::2]
        return float(acc[0]) if len(acc) else 0.0

    for j in range(m - 2, -1, -1):
        cf = cf * disc
        itm = h_all[j] > 0
        yy = y_all[j][itm]
        if yy.size < p:
            continue
        pw = [np.ones_like(yy)]
        for k in range(1, 2 * p - 1):
            pw.append(pw[-1] * yy)
        G = np.array([[fsum(pw[a + b]) for b in range(p)] for a in range(p)])
        beta = oracle.solve_normal(G, np.array([fsum(cf[itm] * pw[k]) for k in range(p)]))
        if beta is None:
            continue
        cont = sum(np.float32(beta[k]) * pw[k] for k in range(p))
        ex = h_all[j][itm] > cont
        c = cf[itm]
        c[ex] = h_all[j][itm][ex]
        cf[itm] = c
    return float(np.exp(-o.r * o.T / m) * np.mean(cf.astype(np.float64)))


def fp32_sum_shift(o):
    S = paths(o)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"] / o.K
    return abs(lsm_fp32_sums(S, o) - ref)


def check_mixed_vs_oracle(o, got, ref, fp64_price, replay, bar=2e-4):
    """A mixed-precision price `got` against the oracle's `ref` on the same
    points: within bar K.  Otherwise the option must be one on which the LSM
    estimator is unstable at FP32 precision (the oracle's own price moves by
    more than half the bar under FP32-level path noise or FP32 sums), and
    then the kernel is held to its arithmetic instead: replay() runs the
    replay check of the mixed sweep on its own FP32 paths (every date's
    normal equations and the price within their FP32 bounds,
    tests/lsm_replay.py), and the FP64 GPU price fp64_price() must be within
    bar K of the oracle."""
    err = abs(got - ref) / o.K
    if err <= bar:
        return
    spread = max(fp32_noise_spread(o), fp32_sum_shift(o))
    assert spread > bar / 2, ("mixed price off the oracle on an FP32-stable option", o, got, ref, spread)
    replay()
    assert abs(fp64_price() - ref) <= bar * o.K, (o, ref)


def binary16_moneyness(S, K):
    """Paths S (FP64) with their moneyness y = S/K - 1 rounded to IEEE
    binary16 (round to nearest even), as prices K (1 + y)."""
    return K * (1.0 + (S / K - 1.0).astype(np.float16).astype(np.float64))


def binary16_shift(o):
    """|oracle price on the binary16-rounded paths - oracle price| / K."""
    S = paths(o)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"]
    return abs(oracle.lsm(binary16_moneyness(S, o.K), o.type, o.K, o.r, o.T, o.basis)["price"] - ref) / o.K


def check_mixed16_vs_oracle(o, got, ref, fp64_price, replay, bar=2e-4):
    """As check_mixed_vs_oracle for the binary16 path array (AMC_MIXED16):
    a price off the oracle by more than bar K is accepted only on an option
    whose oracle price itself moves by more than half the bar when its paths
    are rounded to binary16 moneyness (or under FP32-level noise); the
    kernel is then held to the replay check on its own binary16 paths and
    the FP64 GPU price to bar K."""
    err = abs(got - ref) / o.K
    if err <= bar:
        return
    spread = max(binary16_shift(o), fp32_noise_spread(o))
    assert spread > bar / 2, ("binary16 price off the oracle on a stable option", o, got, ref, spread)
    replay()
    assert abs(fp64_price() - ref) <= bar * o.K, (o, ref)
