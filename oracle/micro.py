"""Second, independent LSM oracle for tiny inputs (numpy; test infrastructure).

Longstaff & Schwartz (ref. [12] of the paper) written a second way: the
regression at each date is an ordinary least-squares fit by
``numpy.linalg.lstsq`` (SVD) instead of equilibrated normal equations, and the
loop keeps whole-array state.  Used only on a handful of paths and dates so
that its per-date coefficients, cash flows and stopping dates can be compared
with the C oracle entry by entry.
"""
import numpy as np


def lsm_micro(S, type_, K, r, T, p, center=1.0):
    """S: (m, N) date-major paths.  Regression basis 1, y, .., y^(p-1) with
    y = S/K - center (center 1: the oracle's moneyness basis; center 0: the
    plain S/K monomials, which span the same functions).  Returns
    dict(price, beta (m,p), tau, cf, degenerate)."""
    S = np.asarray(S, dtype=np.float64)
    m, N = S.shape
    dt = T / m
    disc = np.exp(-r * dt)
    pay = (lambda s: np.maximum(s - K, 0.0)) if type_ == 1 else (lambda s: np.maximum(K - s, 0.0))
    cf = pay(S[m - 1]).copy()
    tau = np.full(N, m, dtype=np.int32)
    beta = np.zeros((m, p))
    degenerate = 0
    for j in range(m - 1, 0, -1):
        cf = cf * disc
        h = pay(S[j - 1])
        itm = np.nonzero(h > 0)[0]
        if itm.size < p:
            degenerate += 1
            continue
        x = S[j - 1, itm] / K - center
        X = np.vander(x, p, increasing=True)
        if np.linalg.matrix_rank(X) < p:
            degenerate += 1
            continue
        b, *_ = np.linalg.lstsq(X, cf[itm], rcond=None)
        beta[j - 1] = b
        ex = itm[h[itm] > X @ b]
        cf[ex] = h[ex]
        tau[ex] = j
    return {"price": disc * cf.mean(), "beta": beta, "tau": tau, "cf": cf, "degenerate_dates": degenerate}


def cash_flows_under_boundary(S, type_, K, r, T, beta, deg):
    """Brute force, one path and one date at a time: the cash flow of each
    path under a given exercise boundary (beta[m, p] in currency units on the
    basis 1, y, .., y^(p-1), y = S/K - 1; deg[m] nonzero = no exercise),
    discounted to t_j before the decision at t_j.  Returns cf[m, N]; row j-1
    is what the regression of date j is fitted to when the later decisions
    are the boundary's (ref. [12])."""
    S = np.asarray(S, dtype=np.float64)
    m, N = S.shape
    disc = np.exp(-r * T / m)
    out = np.zeros((m, N))
    for i in range(N):
        s_m = S[m - 1, i]
        c = max(s_m - K, 0.0) if type_ == 1 else max(K - s_m, 0.0)
        out[m - 1, i] = c
        for j in range(m - 1, 0, -1):
            c = c * disc
            out[j - 1, i] = c
            if deg[j - 1]:
                continue
            s = S[j - 1, i]
            h = max(s - K, 0.0) if type_ == 1 else max(K - s, 0.0)
            if not h > 0.0:
                continue
            y = s / K - 1.0
            cont = sum(beta[j - 1][k] * y ** k for k in range(len(beta[j - 1])))
            if h > cont:
                c = h
    return out
