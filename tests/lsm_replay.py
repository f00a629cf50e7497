"""Replay check of a mixed-precision LSM sweep on its own paths (test helper).

Where the LSM estimator is unstable at FP32 precision (a cubic basis over a
wide moneyness range), exercise decisions near the fitted boundary flip under
perturbations of order 1e-7.  One flip changes the cash flows that every
earlier date regresses on, so a free-running FP32 sweep and the FP64 oracle
drift apart by more than 2e-4 K, and comparing their prices says nothing
about the kernel.  This check instead holds the kernel to the arithmetic it
performs, date by date.

Inputs: the GPU's FP32 paths S (exact values, as float64), and the boundary
the GPU fitted on them (amc_fit_boundary: per date d the FP32 coefficients
beta_d, units of K on the basis 1, y, .., y^(p-1) with y = S/K - 1, and its
degenerate flag).  The oracle then replays the backward induction in FP64 on
the same paths with the GPU's decisions (oracle.value_boundary with
cf_dates): at each date j the cash flows CF_j that the regression of date j
is fitted to, given the decisions at the later dates.  For each date j with
in-the-money set I_j (FP64) the oracle's normal equations are
    G_kl = sum_I y^(k+l),   R_k = sum_I y^k CF_j,
and the GPU's beta_j must satisfy them up to the perturbation that its FP32
arithmetic can introduce (a backward-error bound, with no linearisation and
no condition number):
    |G beta_j - R|_k <= sum_l dG_kl |beta_l| + dR_k + 4u sum_l |G_kl| |beta_l|,
u = 2^-24, where
    dG_kl = 24u sum_I |y|^q + sum_I q |y|^(q-1) dy                 (q = k+l)
            + sum over paths whose in-the-money test is ambiguous of |y|^q,
    dR_k  = 24u sum_I |y|^k |CF| + sum_I |y|^k dCF + sum_I k |y|^(k-1) dy |CF|
            + sum over paths of I whose decision at a later date is ambiguous
              of |y|^k Cmax
            + sum over ambiguous in-the-money paths of |y|^k (|CF| + Cmax).
The terms:
  24u      per sum: a term y^q or y^k CF is formed with up to 3 roundings,
           then passes through at most 10 FP32 additions in its thread (the
           cluster sweep's 8 or 9 packed pairs and the pair's two halves, or
           its one shared-memory path; 8 paths in the L2-exchange sweep), 5
           levels of the warp tree and 5 of the FP32 tree over the CTA's
           warps; the CTAs' totals are added in double-float; 23u < 24u;
  dy       the GPU forms y = fma(S, fl(1/K), -1) in FP32:
           |dy| <= u (1 + 2|y|);
  dCF      the GPU's cash flow is h (from its y) discounted by fl(e^{-r dt})
           once per date in FP32: |dCF| <= (2(m - j) + 4) u |CF| + 2u;
  4u       the FP64 inverse and the double-float product G^-1 R, rounded to
           the FP32 coefficients the path warps use;
  Cmax     the largest cash flow any path can carry (max h, times e^{rT}
           when r < 0): a bound on the change of CF_j when a decision flips.
A decision at date d is ambiguous when |h - c_d(y)| is within
    2 [u (1 + 2|y|)(1 + |c_d'(y)|) + 6u sum_k |beta_k| |y|^k]
(FP32 Horner evaluation by three FMAs on an FP32 y); an in-the-money test is
ambiguous when |y| <= u (1 + 2|y|).  Degenerate flags must agree, except
where an in-the-money test is ambiguous or the smallest pivot of the
equilibrated Cholesky factorisation is below 1e-4 (within reach of FP32
perturbations of the sums, against the 1e-12 threshold).
The price: the GPU's in-sample price against the oracle's FP64 value of the
same paths under the same boundary, within
    K e^{-r dt} [mean((2m + 4)u |CF| + 2u) + 16u mean |CF| + n_flip Cmax / N],
n_flip the paths with an ambiguous decision at any date.

A dropped term, a wrong sign or index in a moment or right-hand side, a
wrong exercise test or a wrong discount makes a residual or the price miss
its bound by orders of magnitude; FP32 rounding cannot.
"""
import math

import numpy as np

import oracle

U = 2.0 ** -24


def gpu_fit(amc, ctx, torch, o, streaming=False, h16=False):
    """The GPU's FP32 paths of option o (exact values as float64 [m, N]), the
    boundary its mixed sweep fits on them ([m, AMC_COEF_STRIDE]) and its
    in-sample result dict; streaming: the streaming sweep of large options
    (forced by amc_ctx_inject kind 3) instead of the register-resident one;
    h16: the binary16 moneyness path array (AMC_MIXED16), returned as the
    prices K (1 + y) in FP64 (the sweep reads y exactly, so the bound on dy
    below holds with room to spare)."""
    ld = amc.amc_path_ld(o.n_paths)
    prec = amc.AMC_MIXED16 if h16 else amc.AMC_MIXED
    S = torch.empty((o.n_steps, ld), dtype=torch.float16 if h16 else torch.float32, device="cuda")
    coef = torch.full((o.n_steps, amc.AMC_COEF_STRIDE), float("nan"), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_generate_paths(ctx, o, prec, S)
    if streaming:
        ctx.inject(3)
    amc.amc_fit_boundary(ctx, o, prec, S, coef, res)
    torch.cuda.synchronize()
    Sh = S[:, :o.n_paths].double().cpu().numpy()
    if h16:
        Sh = o.K * (1.0 + Sh)
    return Sh, coef.cpu().numpy(), amc.res_to_dict(res.cpu().numpy())


def gpu_replay(amc, ctx, o, streaming=False, h16=False):
    """gpu_fit then replay_check: the mixed sweep of o held to its FP32
    arithmetic on its own paths."""
    import torch
    S, coef, res = gpu_fit(amc, ctx, torch, o, streaming=streaming, h16=h16)
    return replay_check(S, o, coef, res)


def _min_pivot(G):
    """Smallest pivot of the Cholesky factorisation of the equilibrated G."""
    d = np.sqrt(np.diag(G))
    if not (d > 0).all():
        return 0.0
    A = G / np.outer(d, d)
    p = len(d)
    L = np.zeros_like(A)
    piv = np.inf
    for k in range(p):
        for l in range(k + 1):
            acc = A[k, l] - L[k, :l] @ L[l, :l]
            if l == k:
                piv = min(piv, acc)
                if acc <= 0:
                    return float(acc)
                L[k, k] = math.sqrt(acc)
            else:
                L[k, l] = acc / L[l, l]
    return float(piv)


def _powers(y, n):
    out = [np.ones_like(y)]
    for _ in range(1, n):
        out.append(out[-1] * y)
    return out


def replay_check(S, o, coef, res):
    """Assert the bounds above for every date and for the price; returns the
    largest residual / bound ratio, the price error / bound ratio and the
    number of ambiguous decisions."""
    m, N = S.shape
    p, K = o.basis, o.K
    put = o.type == oracle.PUT
    assert res["status"] == 0, res
    deg = coef[:, 4] != 0
    assert deg[m - 1]
    beta = np.where(deg[:, None], 0.0, coef[:, :p])
    val = oracle.value_boundary(S, o.type, K, o.r, o.T, beta * K, deg.astype(np.int32), details=True, cf_dates=True)
    cfd = val["cf_dates"] / K
    y = S / K - 1.0
    h = np.maximum(-y if put else y, 0.0)
    disc = math.exp(-o.r * o.T / m)
    Cmax = float(h.max()) * max(1.0, disc ** -m)
    dy = U * (1.0 + 2.0 * np.abs(y))
    amb_itm = np.abs(y) <= dy
    flipped = np.zeros(N, dtype=bool)            # paths with an ambiguous decision at a later date
    worst = 0.0
    n_amb = 0
    for j in range(m - 1, 0, -1):
        row = j - 1
        I = h[row] > 0
        nI = int(I.sum())
        yI, cI = y[row][I], cfd[row][I]
        q_pows = _powers(yI, 2 * p - 1)
        G = np.array([[q_pows[k + l].sum() for l in range(p)] for k in range(p)])
        R = np.array([(q_pows[k] * cI).sum() for k in range(p)])
        orc_deg = nI < p or oracle.solve_normal(G, R) is None
        if deg[row] and not orc_deg:
            # the GPU's pivots come from FP32 sums: a flag may differ only
            # where the smallest equilibrated pivot is within reach of them
            assert amb_itm[row].any() or _min_pivot(G) < 1e-4, ("degenerate flag differs", j, nI, _min_pivot(G))
        if not deg[row]:
            assert nI >= p or amb_itm[row].any(), ("too few in-the-money paths for a fit", j, nI)
            ay = np.abs(yI)
            ap = _powers(ay, 2 * p - 1)
            dyI = dy[row][I]
            ya, ca = np.abs(y[row][amb_itm[row]]), np.abs(cfd[row][amb_itm[row]])
            apa = _powers(ya, 2 * p - 1)
            dM = np.array([24 * U * ap[q].sum() + (q * ap[q - 1] * dyI).sum() if q else 24 * U * nI
                           for q in range(2 * p - 1)])
            dM += np.array([apa[q].sum() for q in range(2 * p - 1)])
            dcf = (2 * (m - j) + 4) * U * np.abs(cI) + 2 * U
            fI = flipped[I]
            dR = np.array([24 * U * (ap[k] * np.abs(cI)).sum() + (ap[k] * dcf).sum()
                           + ((k * ap[k - 1] * dyI * np.abs(cI)).sum() if k else 0.0)
                           + (ap[k][fI] * Cmax).sum() + (apa[k] * (ca + Cmax)).sum() for k in range(p)])
            b = beta[row]
            r = G @ b - R
            bound = (np.array([sum(dM[k + l] * abs(b[l]) for l in range(p)) for k in range(p)]) + dR
                     + 4 * U * (np.abs(G) @ np.abs(b)))
            ratio = float(np.max(np.abs(r) / bound))
            worst = max(worst, ratio)
            assert ratio <= 1.0, ("normal-equation residual beyond the FP32 bound", j, r, bound)
        if not deg[row]:
            b = beta[row]
            yr = y[row]
            ypow = _powers(yr, p)
            c = sum(b[k] * ypow[k] for k in range(p))
            dc = sum(k * b[k] * ypow[k - 1] for k in range(1, p))
            ab = sum(abs(b[k]) * np.abs(ypow[k]) for k in range(p))
            d_eval = 2.0 * (dy[row] * (1.0 + np.abs(dc)) + 6 * U * ab)
            amb = ((h[row] > 0) & (np.abs(h[row] - c) <= d_eval)) | amb_itm[row]
            n_amb += int(amb.sum())
            flipped |= amb
    # price: in-sample GPU price against the FP64 value under the same boundary
    cf_end = np.where(val["tau"] == 1, h[0], cfd[0])
    a = np.abs(cf_end)
    pbound = K * disc * (((2 * m + 4) * U * a + 2 * U).mean() + 16 * U * a.mean() + flipped.sum() * Cmax / N)
    perr = abs(res["price"] - val["price"])
    assert perr <= pbound, ("price beyond the FP32 bound under the GPU's boundary", res["price"], val["price"], pbound)
    return {"residual_ratio": worst, "price_ratio": perr / pbound, "ambiguous": n_amb, "flipped_paths": int(flipped.sum())}
