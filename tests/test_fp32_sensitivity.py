"""Why two GPU parity cases are held to the 2e-4 K bar in FP64 only.

LSM with a cubic basis over a very wide moneyness range (volatility 150 %;
a 10-year call at 40 %) is unstable: exercise decisions near the fitted
boundary flip under perturbations of order 1e-7..1e-5, and each flip feeds the
regressions of all earlier dates.  The mixed path's FP32 paths differ from the
FP64 ones by up to 2e-5 relative and its sweep sums in FP32 before the
double-float stages, so on these cases the oracle's own price moves beyond
the bar under either perturbation, while a stable case stays far inside it.
Written here in numpy from the sweep's definition (oracle paths and solve).
"""
import numpy as np

import oracle
import workloads

STABLE = workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, seed=1)
HUGE_VOL = workloads.Option(100.0, 100.0, 0.05, 1.5, 1.0, 50, 8192, basis=4, seed=21)
LONG_CALL = workloads.Option(50.0, 60.0, 0.08, 0.4, 10.0, 120, 8192, basis=4, type=1, seed=26)


def _paths(o):
    return oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed)


def _path_noise_spread(o, eps=2e-5, reps=4):
    S = _paths(o)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"]
    return max(abs(oracle.lsm(S * (1 + eps * np.random.default_rng(k).standard_normal(S.shape)), o.type, o.K, o.r,
                              o.T, o.basis)["price"] - ref) / o.K for k in range(reps))


def _lsm_fp32_sums(S, o):
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


def _fp32_sum_shift(o):
    S = _paths(o)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)["price"] / o.K
    return abs(_lsm_fp32_sums(S, o) - ref)


def test_stable_case_is_insensitive():
    assert _path_noise_spread(STABLE) < 1e-4          # half the bar
    assert _fp32_sum_shift(STABLE) < 1e-4


def test_wide_range_cubic_cases_are_unstable_at_fp32_precision():
    assert _path_noise_spread(HUGE_VOL) > 2e-4
    assert _path_noise_spread(LONG_CALL) > 2e-4
    assert _fp32_sum_shift(HUGE_VOL) > 1e-4
