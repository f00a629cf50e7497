"""Fit the single-precision inverse-normal polynomials used by pathgen.cu
and dual.cu (icdf.cuh).

Form (the two-region construction of M. Giles, "Approximating the erfinv
function", GPU Computing Gems, 2010, applied to the normal quantile): with
y = u - 1/2, p = min(u, 1-u) and w = -log(4 p (1 - p)),
    z = y * A(w - W0/2)          for |y| < Y0   (w < W0 = 6, 99.88 %)
    z = y * B(sqrt(w) - 3)       otherwise      (tails, down to p = 2^-33)
Y0 is the float just below 1/2 - p(W0), the threshold the kernels test.
A (degree 7) and B (degree 9) are polynomials.  The coefficients here are
this project's own: a Chebyshev least-squares fit, in double precision, to
z/y computed from scipy.special.ndtri, then rounded to float.  The script
prints them, Y0, and the worst relative error of a float32 Horner
evaluation against ndtri over the whole 32-bit uniform grid.

Run: python fit_icdf.py
"""
import numpy as np
from scipy.special import ndtri

W0 = 6.0
DEG_A, DEG_B = 7, 9
S_MAX = np.sqrt(-np.log(4 * 2.0 ** -33 * (1 - 2.0 ** -33))) + 0.05


def p_of_w(w):
    return 0.5 * (1.0 - np.sqrt(-np.expm1(-w)))        # lower-tail p with 4p(1-p) = e^-w


def fit(xs, ys, deg, center):
    c = np.polynomial.chebyshev.chebfit(xs, ys, deg)
    poly = np.polynomial.chebyshev.cheb2poly(c)           # in x
    # re-expand around `center`: coefficients of (x - center)^k
    P = np.polynomial.polynomial
    shifted = np.zeros(deg + 1)
    for k, a in enumerate(poly):
        t = P.polypow([center, 1.0], k)
        shifted[:len(t)] += a * t
    return shifted.astype(np.float32)


def horner32(coef, x):
    x = x.astype(np.float32)
    acc = np.full_like(x, coef[-1], dtype=np.float32)
    for a in coef[-2::-1]:
        acc = (acc.astype(np.float64) * x.astype(np.float64) + np.float64(a)).astype(np.float32)
    return acc


def main():
    y0 = np.float32(0.5 - p_of_w(W0))
    y0 = np.nextafter(y0, np.float32(0)) if y0 > 0.5 - p_of_w(W0) else y0  # at or below 1/2 - p(W0)
    w_lo = -np.log(4 * (0.5 - float(y0)) * (0.5 + float(y0)))               # the tail starts here (<= W0)
    wa = np.cos(np.linspace(np.pi, 0, 4001)) * (W0 / 2) + W0 / 2          # Chebyshev-spaced w in [0, W0]
    wa = wa[wa > 1e-9]
    pa = p_of_w(wa)
    ya = pa - 0.5
    A = fit(wa, ndtri(pa) / ya, DEG_A, W0 / 2)
    s_lo = np.sqrt(w_lo) - 0.01
    sb = np.cos(np.linspace(np.pi, 0, 4001)) * (S_MAX - s_lo) / 2 + (S_MAX + s_lo) / 2
    pb = p_of_w(sb ** 2)
    yb = pb - 0.5
    B = fit(sb, ndtri(pb) / yb, DEG_B, 3.0)
    # float32 check on dense samples across the whole 32-bit uniform grid
    x = np.unique(np.concatenate([np.linspace(0, 2 ** 32 - 1, 2_000_001).astype(np.uint64),
                                  np.arange(0, 2 ** 16, dtype=np.uint64),
                                  (2 ** 32 - 1 - np.arange(0, 2 ** 16, dtype=np.uint64))]))
    u = (x.astype(np.float64) + 0.5) * 2.0 ** -32
    y = u - 0.5
    p = np.minimum(u, 1 - u)
    w = -np.log(4 * p * (1 - p))
    central = np.abs(y.astype(np.float32)) < y0
    z = np.where(central, y * horner32(A, w - W0 / 2), y * horner32(B, np.sqrt(w) - 3.0))
    ref = ndtri(u)
    rel = np.abs(z - ref) / np.maximum(np.abs(ref), 1e-3)
    print("A =", ", ".join("%.9ef" % a for a in A))
    print("B =", ", ".join("%.9ef" % b for b in B))
    print("Y0 = %.9ef" % y0)
    print("central share of the uniform grid %.5f; max rel err %.3e (central %.3e, tail %.3e)" % (
        1.0 - 2.0 * (0.5 - float(y0)), rel.max(), rel[central].max(), rel[~central].max()))


if __name__ == "__main__":
    main()
