"""The streaming LSM sweep's order of operations, restated in numpy on the
oracle's paths and solve, gives the oracle's backward induction: the pass of
date j applies the exercise decision of date j+1 (with the coefficients
solved one pass earlier), discounts the cash flows to t_j, then sums the
moments and right-hand sides of date j; a final pass applies the decision
of date 1.  (CPU; the GPU kernels follow this order and are checked against
the oracle in tests/test_gpu_large.py.)"""
import numpy as np
import pytest

import oracle
import workloads


def _streaming_order(S, K, r, T, p, put):
    m, N = S.shape
    disc = np.exp(-r * T / m)
    y = S / K - 1.0
    h = np.maximum(-y if put else y, 0.0)
    itm = (y < 0) if put else (y > 0)
    beta, deg, cf = {}, {}, None

    def exercise(d):
        b = beta[d]
        yy = y[d - 1]
        cont = ((b[3] * yy + b[2]) * yy + b[1]) * yy + b[0]
        ex = itm[d - 1] & (h[d - 1] > cont)
        cf[ex] = h[d - 1][ex]

    for j in range(m - 1, 0, -1):
        if j == m - 1:
            cf = h[m - 1].copy()
        elif not deg[j + 1]:
            exercise(j + 1)
        cf = cf * disc
        I = itm[j - 1]
        yy, c = y[j - 1][I], cf[I]
        M = [np.sum(yy ** k) for k in range(2 * p - 1)]
        G = np.array([[M[a + b] for b in range(p)] for a in range(p)])
        R = np.array([np.sum(c * yy ** k) for k in range(p)])
        sol = oracle.solve_normal(G, R) if I.sum() >= p else None
        deg[j] = sol is None
        beta[j] = np.zeros(4)
        if sol is not None:
            beta[j][:p] = sol
    if m == 1:
        cf = h[0].copy()
    elif not deg[1]:
        exercise(1)
    return disc * np.mean(cf) * K, sum(deg.values())


CASES = [workloads.single_small(),
         workloads.Option(105.0, 100.0, 0.04, 0.25, 0.75, 7, 12345, basis=2, type=1, seed=11),
         workloads.Option(95.0, 100.0, 0.07, 0.35, 1.5, 30, 3001, basis=4, seed=12),
         workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 1, 999, seed=3),
         workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 2, 999, seed=3),
         workloads.Option(200.0, 40.0, 0.06, 0.2, 1.0, 20, 2000, basis=3, seed=18)]


@pytest.mark.parametrize("o", CASES, ids=["ls_table1", "call_p2", "put_p4", "one_date", "two_dates", "degenerate"])
def test_streaming_order_is_the_oracle_backward_induction(o):
    S = oracle.paths(o.S0, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.seed)
    ref = oracle.lsm(S, o.type, o.K, o.r, o.T, o.basis)
    got, ndeg = _streaming_order(S, o.K, o.r, o.T, o.basis, o.type == oracle.PUT)
    assert got == pytest.approx(ref["price"], rel=1e-12, abs=1e-12 * o.K)
    assert ndeg == ref["degenerate_dates"]
