"""FP64 CPU oracle for the QMC American-option hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg and the reference arm of bench.py, never by the product
library.  It shares no
code with the CUDA path.  The arithmetic lives in ``amc_oracle.c`` (plain C,
double precision, written step by step after the paper); this module only
marshals numpy arrays into it and reads the raw Joe-Kuo data (primitive
polynomials and initial direction numbers, Joe & Kuo 2008) from the data file
that ships with scipy.

Functions and the passages they follow:
  shifts         digital shift per dimension, SplitMix64(seed) high words
  directions     Sobol' direction numbers (Bratley-Fox recurrence)
  sobol          32-bit Sobol' integers, Gray-code order (§III.D)
  norm_icdf      inverse cumulative normal as the root of Phi(z)=u (§III.D)
  bridge_schedule breadth-first Brownian-bridge bisection (ref. [13])
  paths          steps 1-3: points -> normals -> bridge -> GBM (Eq. 9)
  lsm            Longstaff-Schwartz sweep (ref. [12], §V backward induction)
  paper_ub       the paper's exercise rule, Eqs. 10-11
  european       Eqs. 6-8
  bs             Black-Scholes, Eqs. 1-5
  crr            Cox-Ross-Rubinstein tree (Bermudan or American)
  pathwise_greeks frozen-boundary pathwise delta and vega
  solve_normal   equilibrated Cholesky solve of one date's normal equations
  price, greeks  the above from option parameters (points, paths, rule)
  lcg_params, lcg_perm, paths_permuted
                 the paper's LCG-permuted points (§III.D)
  value_boundary, price_oos
                 a fitted boundary applied to other paths (second pass,
                 ref. [12])
  dual_normal, dual_upper, price_dual
                 Andersen-Broadie dual upper bound of a fitted boundary
                 (§IV, ref. [11])
  bridge_matrix  the bridge as a linear map W = A z (for the covariance pin)
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None
PUT, CALL = 0, 1
RULE_LSM, RULE_PAPER_UB, RULE_EUROPEAN = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_ip = ctypes.POINTER(ctypes.c_int)


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        lib.orc_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.orc_splitmix64_next.restype = ctypes.c_uint64
        lib.orc_digital_shifts.argtypes = [ctypes.c_uint64, ctypes.c_int, _u32p]
        lib.orc_sobol_directions.argtypes = [ctypes.c_int, _i64p, _i64p, ctypes.c_int, _u32p]
        lib.orc_sobol_direct.argtypes = [_u32p, ctypes.c_int, ctypes.c_uint64]
        lib.orc_sobol_direct.restype = ctypes.c_uint32
        lib.orc_sobol_block.argtypes = [_u32p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, _u32p]
        lib.orc_norm_cdf.argtypes = [ctypes.c_double]
        lib.orc_norm_cdf.restype = ctypes.c_double
        lib.orc_norm_icdf.argtypes = [ctypes.c_double]
        lib.orc_norm_icdf.restype = ctypes.c_double
        lib.orc_uniform.argtypes = [ctypes.c_uint32]
        lib.orc_uniform.restype = ctypes.c_double
        lib.orc_bridge_schedule.argtypes = [ctypes.c_int, _ip, _ip, _ip]
        lib.orc_paths.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _u32p, _u32p,
                                                          _dp, _dp]
        lib.orc_lcg_modulus.argtypes = [ctypes.c_int64]
        lib.orc_lcg_modulus.restype = ctypes.c_uint64
        lib.orc_lcg_params.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, _u64p, _u64p]
        lib.orc_lcg_perm.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                     ctypes.c_uint64]
        lib.orc_lcg_perm.restype = ctypes.c_uint64
        lib.orc_paths_permuted.argtypes = ([ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_int64, _u32p, _u64p, _u64p,
                                                                    _dp])
        lib.orc_dual_normal.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                        ctypes.c_int64, ctypes.c_int]
        lib.orc_dual_normal.restype = ctypes.c_double
        lib.orc_dual_upper.argtypes = ([ctypes.c_int] + [ctypes.c_double] * 4 +
                                       [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _dp, _dp, _i32p, ctypes.c_int64,
                                        ctypes.c_uint64, _dp, _dp])
        lib.orc_bs.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5
        lib.orc_bs.restype = ctypes.c_double
        lib.orc_solve_normal.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        lib.orc_lsm.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, _i32p, _dp, _i64p, _i32p]
        lib.orc_value_boundary.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int64, ctypes.c_int, _dp, _dp, _i32p, _dp, _i32p,
                                           _dp]
        lib.orc_paper_ub.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int64, _dp, _dp]
        lib.orc_european.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.c_int64, _dp, _dp]
        lib.orc_pathwise_greeks.argtypes = ([ctypes.c_int] + [ctypes.c_double] * 5 +
                                            [ctypes.c_int, ctypes.c_int64, _dp, _dp, _i32p, _dp])
        lib.orc_crr.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5 + [ctypes.c_int] * 3
        lib.orc_crr.restype = ctypes.c_double
        lib.orc_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        _LIB = lib
    return _LIB


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


# ----------------------------------------------------------------------------
def joe_kuo_raw(m):
    """Raw Joe-Kuo data for dimensions 0..m-1: (poly int64[m], vinit int64[m,18])."""
    import scipy.stats
    path = os.path.join(os.path.dirname(scipy.stats.__file__), "_sobol_direction_numbers.npz")
    with np.load(path) as d:
        poly = np.ascontiguousarray(d["poly"][:m], dtype=np.int64)
        vinit = np.ascontiguousarray(d["vinit"][:m], dtype=np.int64)
    if poly.shape[0] < m:
        raise ValueError("Joe-Kuo data holds %d dimensions, %d asked" % (poly.shape[0], m))
    return poly, vinit


def threads():
    """Threads the oracle's OpenMP loops use."""
    return _lib().orc_threads()


def set_threads(n):
    """Sets the threads of the oracle's OpenMP loops."""
    _lib().orc_set_threads(int(n))


def splitmix64(seed, n):
    st = ctypes.c_uint64(seed)
    return [_lib().orc_splitmix64_next(ctypes.byref(st)) for _ in range(n)]


def shifts(seed, m):
    out = np.zeros(m, dtype=np.uint32)
    _lib().orc_digital_shifts(ctypes.c_uint64(seed), m, _ptr(out, _u32p))
    return out


def directions(m):
    poly, vinit = joe_kuo_raw(m)
    V = np.zeros((m, 32), dtype=np.uint32)
    rc = _lib().orc_sobol_directions(m, _ptr(poly, _i64p), _ptr(vinit, _i64p), vinit.shape[1], _ptr(V, _u32p))
    if rc != 0:
        raise ValueError("direction-number expansion failed (%d)" % rc)
    return V


def sobol(n, m, i0=0, seed=None, V=None):
    """Unshifted (seed None) or shifted Sobol' integers, shape (m, n), points i0..i0+n-1."""
    if V is None:
        V = directions(m)
    X = np.zeros((m, n), dtype=np.uint32)
    _lib().orc_sobol_block(_ptr(V, _u32p), m, ctypes.c_uint64(i0), n, _ptr(X, _u32p))
    if seed is not None:
        X ^= shifts(seed, m)[:, None]
    return X


def sobol_direct(V, d, i):
    return _lib().orc_sobol_direct(_ptr(V, _u32p), d, ctypes.c_uint64(i))


def norm_icdf(u):
    f = _lib().orc_norm_icdf
    return np.array([f(float(x)) for x in np.ravel(u)]).reshape(np.shape(u))


def norm_cdf(x):
    f = _lib().orc_norm_cdf
    return np.array([f(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def uniform(x):
    f = _lib().orc_uniform
    return np.array([f(int(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def bridge_schedule(m):
    date = np.zeros(m, dtype=np.intc)
    left = np.zeros(m, dtype=np.intc)
    right = np.zeros(m, dtype=np.intc)
    if _lib().orc_bridge_schedule(m, _ptr(date, _ip), _ptr(left, _ip), _ptr(right, _ip)) != 0:
        raise ValueError("bridge schedule failed")
    return date, left, right


def paths(S0, r, sigma, T, m, N, seed, with_W=False, first=0):
    """Steps 1-3: S of shape (m, N), S[j-1, i] = S_{first+i}(t_j); optionally W too."""
    V = directions(m)
    sh = shifts(seed, m)
    S = np.empty((m, N), dtype=np.float64)
    W = np.empty((m, N), dtype=np.float64) if with_W else None
    rc = _lib().orc_paths(S0, r, sigma, T, m, N, first, _ptr(V, _u32p), _ptr(sh, _u32p), _ptr(S, _dp), _ptr(W, _dp))
    if rc != 0:
        raise MemoryError("oracle path generation failed (%d)" % rc)
    return (S, W) if with_W else S


def lcg_params(seed, m, N):
    """Per-dimension (a_d, c_d) and the modulus M of the paper's LCG permutation."""
    a = np.zeros(m, dtype=np.uint64)
    c = np.zeros(m, dtype=np.uint64)
    _lib().orc_lcg_params(seed, m, N, _ptr(a, _u64p), _ptr(c, _u64p))
    return a, c, int(_lib().orc_lcg_modulus(N))


def lcg_perm(seed, d, N, i):
    """pi_d(i) for the points 0..N-1 (vectorised over i with a Python loop)."""
    a, c, M = lcg_params(seed, d + 1, N)
    f = _lib().orc_lcg_perm
    return np.array([f(int(a[d]), int(c[d]), M, N, int(k)) for k in np.atleast_1d(i)], dtype=np.int64)


def paths_permuted(S0, r, sigma, T, m, N, seed):
    """Steps 1-3 with the paper's LCG permutation of each dimension's
    (unshifted) quasi-random array instead of the digital shift."""
    V = directions(m)
    a, c, _ = lcg_params(seed, m, N)
    S = np.empty((m, N), dtype=np.float64)
    rc = _lib().orc_paths_permuted(S0, r, sigma, T, m, N, _ptr(V, _u32p), _ptr(a, _u64p), _ptr(c, _u64p),
                                   _ptr(S, _dp))
    if rc != 0:
        raise MemoryError("oracle permuted path generation failed (%d)" % rc)
    return S


def bs(type_, S, K, r, sigma, T):
    return _lib().orc_bs(type_, S, K, r, sigma, T)


def solve_normal(G, b):
    p = len(b)
    G = np.ascontiguousarray(G, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    beta = np.zeros(p)
    rc = _lib().orc_solve_normal(p, _ptr(G, _dp), _ptr(b, _dp), _ptr(beta, _dp))
    return (None if rc else beta)


def lsm(S, type_, K, r, T, p, details=False):
    S = np.ascontiguousarray(S, dtype=np.float64)
    m, N = S.shape
    out = np.zeros(3)
    beta = np.zeros((m, p)) if details else None
    tau = np.zeros(N, dtype=np.int32) if details else None
    cf = np.zeros(N) if details else None
    nitm = np.zeros(m, dtype=np.int64) if details else None
    deg = np.zeros(m, dtype=np.int32) if details else None
    rc = _lib().orc_lsm(type_, K, r, T, m, N, p, _ptr(S, _dp), _ptr(out, _dp), _ptr(beta, _dp),
                        _ptr(tau, _i32p), _ptr(cf, _dp), _ptr(nitm, _i64p), _ptr(deg, _i32p))
    if rc != 0:
        raise ValueError("oracle lsm failed")
    res = {"price": out[0], "std_err": out[1], "degenerate_dates": int(out[2])}
    if details:
        res.update(beta=beta, tau=tau, cf=cf, n_itm=nitm, deg=deg)
    return res


def value_boundary(S, type_, K, r, T, beta, deg, details=False, cf_dates=False):
    """Value the paths S with a given exercise boundary: beta[m, p] in
    currency units on the basis (1, y, .., y^(p-1)), y = S/K - 1; deg[m]
    nonzero = no exercise at that date.  cf_dates: also return "cf_dates"
    [m, N], the cash flow of each path under the boundary discounted to t_j
    before the decision at t_j (row j-1), which is what the regression of
    date j is fitted to when the later decisions are the boundary's."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    m, N = S.shape
    p = beta.shape[1]
    out = np.zeros(3)
    tau = np.zeros(N, dtype=np.int32) if details else None
    cfd = np.zeros((m, N)) if cf_dates else None
    rc = _lib().orc_value_boundary(type_, K, r, T, m, N, p, _ptr(S, _dp), _ptr(beta, _dp), _ptr(deg, _i32p),
                                   _ptr(out, _dp), _ptr(tau, _i32p), _ptr(cfd, _dp))
    if rc != 0:
        raise ValueError("oracle value_boundary failed")
    res = {"price": out[0], "std_err": out[1], "degenerate_dates": int(out[2])}
    if details:
        res["tau"] = tau
    if cf_dates:
        res["cf_dates"] = cfd
    return res


def dual_normal(seed_in, m, n_in, i, j, k, s):
    """Normal of inner step s of inner path k from date j of outer path i."""
    return _lib().orc_dual_normal(seed_in, m, n_in, i, j, k, s)


def dual_upper(S, type_, K, r, sigma, T, beta, deg, n_in, seed_in, details=False):
    """Andersen-Broadie dual upper bound on the outer paths S for the boundary
    (beta [m, p] in currency units, deg [m]); returns upper, std_err, L0."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    m, N = S.shape
    out = np.zeros(3)
    U = np.zeros(N) if details else None
    rc = _lib().orc_dual_upper(type_, K, r, sigma, T, m, N, beta.shape[1], _ptr(S, _dp), _ptr(beta, _dp),
                               _ptr(deg, _i32p), n_in, seed_in, _ptr(out, _dp), _ptr(U, _dp))
    if rc != 0:
        raise ValueError("oracle dual_upper failed")
    res = {"upper": out[0], "std_err": out[1], "L0": out[2]}
    if details:
        res["U"] = U
    return res


def price_dual(S0, K, r, sigma, T, n_steps, n_fit, n_outer, n_in, basis=3, type=PUT, seed=0, outer_seed=1,
               seed_in=2):
    """Boundary fitted on the points of `seed` (n_fit paths); on the n_outer
    paths of outer_seed: the lower bound (the boundary applied) and the dual
    upper bound with n_in inner paths per outer path and date."""
    fit = lsm(paths(S0, r, sigma, T, n_steps, n_fit, seed), type, K, r, T, basis, details=True)
    So = paths(S0, r, sigma, T, n_steps, n_outer, outer_seed)
    low = value_boundary(So, type, K, r, T, fit["beta"], fit["deg"])
    up = dual_upper(So, type, K, r, sigma, T, fit["beta"], fit["deg"], n_in, seed_in)
    return fit, low, up


def price_oos(S0, K, r, sigma, T, n_steps, n_paths, basis=3, type=PUT, seed=0, value_seed=1):
    """Out-of-sample LSM: boundary fitted on the points of `seed`, applied to
    the independent points of `value_seed`.  Returns (fit result with beta
    and deg, valuation result)."""
    fit = lsm(paths(S0, r, sigma, T, n_steps, n_paths, seed), type, K, r, T, basis, details=True)
    val = value_boundary(paths(S0, r, sigma, T, n_steps, n_paths, value_seed), type, K, r, T, fit["beta"],
                         fit["deg"])
    return fit, val


def paper_ub(S, type_, S0, K, r, sigma, T):
    S = np.ascontiguousarray(S, dtype=np.float64)
    m, N = S.shape
    out = np.zeros(3)
    _lib().orc_paper_ub(type_, S0, K, r, sigma, T, m, N, _ptr(S, _dp), _ptr(out, _dp))
    return {"price": out[0], "std_err": out[1], "degenerate_dates": 0}


def paper_ub_m1(type_, S0, K, r, sigma, T):
    """m = 1 needs no paths: max(h(S0), BS(S0, K, T))."""
    out = np.zeros(3)
    S = np.zeros(1)
    _lib().orc_paper_ub(type_, S0, K, r, sigma, T, 1, 1, _ptr(S, _dp), _ptr(out, _dp))
    return out[0]


def european(S, type_, K, r, T):
    S = np.ascontiguousarray(S, dtype=np.float64)
    m, N = S.shape
    out = np.zeros(3)
    _lib().orc_european(type_, K, r, T, m, N, _ptr(S, _dp), _ptr(out, _dp))
    return {"price": out[0], "std_err": out[1], "degenerate_dates": 0}


def pathwise_greeks(S, W, tau, type_, S0, K, r, sigma, T):
    S = np.ascontiguousarray(S, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.int32)
    m, N = S.shape
    out = np.zeros(3)
    rc = _lib().orc_pathwise_greeks(type_, S0, K, r, sigma, T, m, N, _ptr(S, _dp), _ptr(W, _dp),
                                    _ptr(tau, _i32p), _ptr(out, _dp))
    if rc != 0:
        raise ValueError("bad tau")
    return {"price": out[0], "delta": out[1], "vega": out[2]}


def crr(type_, S0, K, r, sigma, T, n, m=1, bermudan=False):
    return _lib().orc_crr(type_, S0, K, r, sigma, T, n, m, 1 if bermudan else 0)


# ----------------------------------------------------------------------------
def price(S0, K, r, sigma, T, n_steps, n_paths, basis=3, type=PUT, seed=0, rule=RULE_LSM, details=False):
    """Full oracle pricing of one option on its own Sobol' points."""
    S = paths(S0, r, sigma, T, n_steps, n_paths, seed)
    if rule == RULE_LSM:
        return lsm(S, type, K, r, T, basis, details=details)
    if rule == RULE_PAPER_UB:
        return paper_ub(S, type, S0, K, r, sigma, T)
    if rule == RULE_EUROPEAN:
        return european(S, type, K, r, T)
    raise ValueError("unknown rule")


def greeks(S0, K, r, sigma, T, n_steps, n_paths, basis=3, type=PUT, seed=0, rule=RULE_LSM):
    """Frozen-boundary pathwise price, delta and vega on the oracle's paths."""
    S, W = paths(S0, r, sigma, T, n_steps, n_paths, seed, with_W=True)
    if rule == RULE_LSM:
        tau = lsm(S, type, K, r, T, basis, details=True)["tau"]
    elif rule == RULE_EUROPEAN:
        tau = np.full(n_paths, n_steps, dtype=np.int32)
    else:
        raise ValueError("greeks are defined for the LSM and European rules")
    return pathwise_greeks(S, W, tau, type, S0, K, r, sigma, T)


def bridge_matrix(m, T):
    """W = A z for one path; A[j-1, k] = weight of coordinate k on W(t_j)."""
    A = np.zeros((m, m))
    lib = _lib()
    lib.orc_bridge_matrix.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
    if lib.orc_bridge_matrix(m, T, _ptr(A, _dp)) != 0:
        raise ValueError("bridge matrix failed")
    return A
