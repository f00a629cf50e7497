"""Python binding of the amc C ABI (include/amc.h): GB300 quasi-Monte Carlo
American-option pricing after Cvetanoska & Stojanovski.

Argument marshalling only.  Every step of the hot path (Sobol' points,
inverse normal, Brownian bridge, GBM store, backward sweep, final sums) runs
in the library's CUDA kernels; PyTorch is used for device memory and streams
only.  There is no CPU fallback: if ``libamc.so`` is missing or cannot be
loaded, importing the library raises.

The functions carry the C names.  Options are ``workloads.Option``-like
objects (attributes S0, K, r, sigma, T, n_steps, n_paths, basis, type, seed,
rule) or dicts with those keys.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamc.so")

AMC_OK, AMC_EINVAL, AMC_ENOMEM, AMC_ECUDA, AMC_ETIMEOUT, AMC_EBUSY, AMC_PENDING, AMC_ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7
AMC_ECANCELED = -8
AMC_PUT, AMC_CALL = 0, 1
AMC_RULE_LSM, AMC_RULE_PAPER_UB, AMC_RULE_EUROPEAN = 0, 1, 2
AMC_FP64, AMC_MIXED, AMC_MIXED16 = 0, 1, 2
AMC_RES_DOUBLES = 8
AMC_COEF_STRIDE = 5
AMC_DUAL_MAX_WORK = 1 << 40
AMC_DUAL_MAX_INNER = 1 << 29
AMC_MAX_STEPS = 512


class amc_option(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("K", ctypes.c_double), ("r", ctypes.c_double),
                ("sigma", ctypes.c_double), ("T", ctypes.c_double), ("n_steps", ctypes.c_int32),
                ("basis", ctypes.c_int32), ("n_paths", ctypes.c_int64), ("type", ctypes.c_int32),
                ("rule", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class amc_result(ctypes.Structure):
    _fields_ = [("price", ctypes.c_double), ("std_err", ctypes.c_double), ("delta", ctypes.c_double),
                ("vega", ctypes.c_double), ("degenerate_dates", ctypes.c_int32), ("status", ctypes.c_int32),
                ("ms_gen", ctypes.c_float), ("ms_sweep", ctypes.c_float)]


class amc_serve_config(ctypes.Structure):
    _fields_ = [("slot_bytes", ctypes.c_size_t), ("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("max_pending", ctypes.c_int32), ("prec", ctypes.c_int32)]


class amc_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("launched", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("batches", ctypes.c_int64), ("pending", ctypes.c_int64),
                ("cancelled", ctypes.c_int64)]


class AmcError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_dp = ctypes.POINTER(ctypes.c_double)
_optp = ctypes.POINTER(amc_option)
_resp = ctypes.POINTER(amc_result)

# name -> (restype, argtypes); the exported surface of include/amc.h
SIGNATURES = {
    "amc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "amc_version": (ctypes.c_int, []),
    "amc_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "amc_ctx_destroy": (ctypes.c_int, [_vp]),
    "amc_ctx_set_timeout": (ctypes.c_int, [_vp, ctypes.c_double]),
    "amc_ctx_inject": (ctypes.c_int, [_vp, ctypes.c_int, _i64]),
    "amc_ctx_memory": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "amc_ctx_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "amc_ctx_profile": (ctypes.c_int, [_vp, _dp, _dp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                       ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "amc_validate_option": (ctypes.c_int, [_optp]),
    "amc_path_ld": (_i64, [_i64]),
    "amc_path_bytes": (ctypes.c_size_t, [ctypes.c_int, _i64, ctypes.c_int]),
    "amc_digital_shifts": (ctypes.c_int, [_u64, ctypes.c_int, _u32p]),
    "amc_sobol_directions": (ctypes.c_int, [ctypes.c_int, _u32p]),
    "amc_bridge_schedule": (ctypes.c_int, [ctypes.c_int, _i32p, _i32p, _i32p]),
    "amc_bridge_plan": (ctypes.c_int, [ctypes.c_int, _i32p, _i32p, _i32p, _i32p, _i32p, _dp, _dp, _dp, _i32p]),
    "amc_plan_sweep": (ctypes.c_int, [_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p]),
    "amc_sobol": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _u64, _vp, _i64, _vp]),
    "amc_generate_paths": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp]),
    "amc_sweep": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, ctypes.c_int, _vp, _vp]),
    "amc_price_device": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp, _vp]),
    "amc_generate_paths_permuted": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp]),
    "amc_lcg_params": (ctypes.c_int, [_u64, ctypes.c_int, _i64, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "amc_fit_boundary": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp, _vp, _vp]),
    "amc_value_boundary": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp, _vp, _vp]),
    "amc_price_oos": (ctypes.c_int, [_vp, _optp, _u64, ctypes.c_int, _resp, _resp]),
    "amc_price_fused": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _vp, _vp]),
    "amc_dual_upper": (ctypes.c_int, [_vp, _optp, ctypes.c_int, _vp, _i64, _vp, _i64, _u64, _vp, _vp, _vp]),
    "amc_price_dual": (ctypes.c_int, [_vp, _optp, _u64, _i64, _i64, _u64, ctypes.c_int, _resp, _resp, _resp]),
    "amc_price_american": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, _i64, ctypes.c_int, ctypes.c_int, _u64,
                                          ctypes.c_int, ctypes.c_int, _resp]),
    "amc_price_batch": (ctypes.c_int, [_vp, _optp, ctypes.c_int, ctypes.c_int, _resp]),
    "amc_greeks": (ctypes.c_int, [_vp, _optp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]),
    "amc_price_batch_device": (ctypes.c_int, [_vp, _optp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "amc_greeks_device": (ctypes.c_int, [_vp, _optp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                         _vp]),
    "amc_serve_start": (ctypes.c_int, [_vp, ctypes.POINTER(amc_serve_config)]),
    "amc_serve_submit": (ctypes.c_int, [_vp, _optp, ctypes.POINTER(_u64)]),
    "amc_serve_poll": (ctypes.c_int, [_vp, _u64, _resp, _dp]),
    "amc_serve_drain": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), _resp, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "amc_serve_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(amc_serve_stats)]),
    "amc_serve_cancel": (ctypes.c_int, [_vp, _u64]),
    "amc_serve_stop": (ctypes.c_int, [_vp]),
    "amc_sweep_noalloc": (ctypes.c_int, [_optp, ctypes.c_int, _vp, _i64, ctypes.c_int, _vp, _vp]),
    "amc_sweep_noalloc_capacity": (ctypes.c_size_t, []),
}


def lib():
    """The loaded libamc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libamc.so not built at %s: run __graft_entry__.build() or "
                              "python paper_1205_0106_gb300/build.py" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().amc_strerror(code).decode()


def _check(rc, what):
    if rc != AMC_OK:
        raise AmcError(rc, what)
    return rc


def _get(o, k):
    return o[k] if isinstance(o, dict) else getattr(o, k)


def make_option(o):
    """amc_option from an Option-like object or dict."""
    if isinstance(o, amc_option):
        return o
    return amc_option(float(_get(o, "S0")), float(_get(o, "K")), float(_get(o, "r")), float(_get(o, "sigma")),
                      float(_get(o, "T")), int(_get(o, "n_steps")), int(_get(o, "basis")), int(_get(o, "n_paths")),
                      int(_get(o, "type")), int(_get(o, "rule")), int(_get(o, "seed")))


def _res_dict(r):
    return {"price": r.price, "std_err": r.std_err, "delta": r.delta, "vega": r.vega,
            "degenerate_dates": r.degenerate_dates, "status": r.status, "ms_gen": r.ms_gen,
            "ms_sweep": r.ms_sweep}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(s):
    if s is None:
        return None
    return ctypes.c_void_p(s.cuda_stream if hasattr(s, "cuda_stream") else int(s))


# ------------------------------------------------------------ host helpers
def amc_version():
    return lib().amc_version()


def amc_validate_option(o):
    return lib().amc_validate_option(ctypes.byref(make_option(o)))


def amc_path_ld(n_paths):
    return lib().amc_path_ld(n_paths)


def amc_path_bytes(n_steps, n_paths, prec):
    return lib().amc_path_bytes(n_steps, n_paths, prec)


def amc_digital_shifts(seed, n_dims):
    import numpy as np
    out = np.zeros(n_dims, dtype=np.uint32)
    _check(lib().amc_digital_shifts(seed, n_dims, out.ctypes.data_as(_u32p)), "amc_digital_shifts")
    return out


def amc_sobol_directions(n_dims):
    import numpy as np
    out = np.zeros((n_dims, 32), dtype=np.uint32)
    _check(lib().amc_sobol_directions(n_dims, out.ctypes.data_as(_u32p)), "amc_sobol_directions")
    return out


def amc_bridge_schedule(n_steps):
    import numpy as np
    d, l, r = (np.zeros(n_steps, dtype=np.int32) for _ in range(3))
    _check(lib().amc_bridge_schedule(n_steps, d.ctypes.data_as(_i32p), l.ctypes.data_as(_i32p),
                                     r.ctypes.data_as(_i32p)), "amc_bridge_schedule")
    return d, l, r


def amc_bridge_plan(n_steps):
    """The depth-first evaluation plan of the bridge: a dict of per-node arrays
    (coord, date, sl, sr, so, wl, wr, sdu) and the slot count n_slots."""
    import numpy as np
    n = max(1, min(n_steps, AMC_MAX_STEPS))             # the library rejects n_steps outside 1..AMC_MAX_STEPS
    ints = {k: np.zeros(n, dtype=np.int32) for k in ("coord", "date", "sl", "sr", "so")}
    dbls = {k: np.zeros(n, dtype=np.float64) for k in ("wl", "wr", "sdu")}
    ns = ctypes.c_int32()
    _check(lib().amc_bridge_plan(n_steps, *(ints[k].ctypes.data_as(_i32p) for k in ("coord", "date", "sl", "sr", "so")),
                                 *(dbls[k].ctypes.data_as(_dp) for k in ("wl", "wr", "sdu")), ctypes.byref(ns)),
           "amc_bridge_plan")
    return dict(**ints, **dbls, n_slots=ns.value)


def amc_plan_sweep(n_paths, sm_count, prec=AMC_MIXED, rule=AMC_RULE_LSM):
    c, p = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().amc_plan_sweep(n_paths, sm_count, prec, rule, ctypes.byref(c), ctypes.byref(p)), "amc_plan_sweep")
    return c.value, p.value


# ------------------------------------------------------------ context
class Context:
    """An amc_ctx on one CUDA device (arena_bytes 0 = 60% of free memory)."""

    def __init__(self, device=0, arena_bytes=0):
        h = ctypes.c_void_p()
        _check(lib().amc_ctx_create(device, arena_bytes, ctypes.byref(h)), "amc_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().amc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_timeout(self, seconds):
        _check(lib().amc_ctx_set_timeout(self.handle, seconds), "amc_ctx_set_timeout")

    def inject(self, kind, arg=0):
        _check(lib().amc_ctx_inject(self.handle, kind, arg), "amc_ctx_inject")

    def set_profiling(self, enable=True):
        _check(lib().amc_ctx_set_profiling(self.handle, 1 if enable else 0), "amc_ctx_set_profiling")

    def profile(self):
        """Device time (ms), launches and path-steps of the path-generation
        and sweep launches since the previous call (profiling on)."""
        g, s = ctypes.c_double(), ctypes.c_double()
        n = [_i64() for _ in range(4)]
        _check(lib().amc_ctx_profile(self.handle, ctypes.byref(g), ctypes.byref(s), *[ctypes.byref(x) for x in n]),
               "amc_ctx_profile")
        return {"gen_ms": g.value, "sweep_ms": s.value, "gen_launches": n[0].value, "sweep_launches": n[1].value,
                "gen_path_steps": n[2].value, "sweep_path_steps": n[3].value}

    def memory(self):
        f, t = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().amc_ctx_memory(self.handle, ctypes.byref(f), ctypes.byref(t)), "amc_ctx_memory")
        return f.value, t.value


def amc_ctx_create(device=0, arena_bytes=0):
    return Context(device, arena_bytes)


def amc_ctx_destroy(ctx):
    ctx.close()


# ------------------------------------------------------------ step level
def amc_sobol(ctx, n_dims, n_points, seed, x, ld=None, stream=None):
    """Shifted Sobol' integers into the uint32-viewed int32 tensor x[n_dims, ld]."""
    ld = x.shape[1] if ld is None else ld
    _check(lib().amc_sobol(ctx.handle, n_dims, n_points, seed, _ptr(x), ld, _stream(stream)), "amc_sobol")


def amc_generate_paths(ctx, opt, prec, S, ld=None, stream=None):
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_generate_paths(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld,
                                    _stream(stream)), "amc_generate_paths")


def amc_sweep(ctx, opt, prec, S, res, ld=None, with_greeks=False, stream=None):
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_sweep(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld, 1 if with_greeks else 0,
                           _ptr(res), _stream(stream)), "amc_sweep")


def amc_price_device(ctx, opt, prec, S, res, ld=None, stream=None):
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_price_device(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld, _ptr(res),
                                  _stream(stream)), "amc_price_device")


def amc_generate_paths_permuted(ctx, opt, prec, S, ld=None, stream=None):
    """Paths from the paper's LCG-permuted (unshifted) quasi-random points."""
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_generate_paths_permuted(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld,
                                             _stream(stream)), "amc_generate_paths_permuted")


def amc_lcg_params(seed, n_dims, n_points):
    """(a[n_dims], c[n_dims], M) of the LCG permutation (host only)."""
    import numpy as np
    a = np.zeros(n_dims, dtype=np.uint32)
    c = np.zeros(n_dims, dtype=np.uint32)
    M = ctypes.c_uint64(0)
    _check(lib().amc_lcg_params(seed, n_dims, n_points, a.ctypes.data_as(_vp), c.ctypes.data_as(_vp),
                                ctypes.byref(M)), "amc_lcg_params")
    return a, c, M.value


def amc_fit_boundary(ctx, opt, prec, S, coef, res, ld=None, stream=None):
    """LSM sweep on S that also writes the fitted boundary into coef
    (device, [n_steps, AMC_COEF_STRIDE] doubles)."""
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_fit_boundary(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld, _ptr(coef),
                                  _ptr(res), _stream(stream)), "amc_fit_boundary")


def amc_value_boundary(ctx, opt, prec, S, coef, res, ld=None, stream=None):
    """Value the paths S with the boundary coef (no regression)."""
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_value_boundary(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld, _ptr(coef),
                                    _ptr(res), _stream(stream)), "amc_value_boundary")


def amc_price_oos(ctx, opt, value_seed, prec=AMC_MIXED):
    """Out-of-sample price: boundary fitted on opt's points, applied to the
    points of value_seed.  Returns (fit result, value result) dicts."""
    fit, val = amc_result(), amc_result()
    _check(lib().amc_price_oos(ctx.handle, ctypes.byref(make_option(opt)), value_seed, prec, ctypes.byref(fit),
                               ctypes.byref(val)), "amc_price_oos")
    return _res_dict(fit), _res_dict(val)


def amc_price_fused(ctx, opt, prec, res, coef=None, stream=None):
    """Steps 1-4 without a path array: the paper's rule or the European
    estimator, or (LSM) the valuation of the boundary coef on opt's points."""
    _check(lib().amc_price_fused(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(coef), _ptr(res),
                                 _stream(stream)), "amc_price_fused")


def amc_dual_upper(ctx, opt, prec, S, coef, n_inner, inner_seed, res, U=None, ld=None, stream=None):
    """Dual upper bound of the boundary coef on the outer paths S: res =
    [mean U, std_err, 0, 0, flagged dates, status, L0, inner steps]; U (device, may
    be None) receives the per-path upper values."""
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_dual_upper(ctx.handle, ctypes.byref(make_option(opt)), prec, _ptr(S), ld, _ptr(coef), n_inner,
                                inner_seed, _ptr(res), _ptr(U), _stream(stream)), "amc_dual_upper")


def amc_price_dual(ctx, opt, outer_seed, n_outer, n_inner, inner_seed, prec=AMC_MIXED):
    """Boundary fitted on opt's points; on n_outer paths of outer_seed its
    value (lower bound) and its dual upper bound.  Returns (fit, lower,
    upper) result dicts."""
    fit, low, up = amc_result(), amc_result(), amc_result()
    _check(lib().amc_price_dual(ctx.handle, ctypes.byref(make_option(opt)), outer_seed, n_outer, n_inner,
                                inner_seed, prec, ctypes.byref(fit), ctypes.byref(low), ctypes.byref(up)),
           "amc_price_dual")
    return _res_dict(fit), _res_dict(low), _res_dict(up)


# ------------------------------------------------------------ serving
def amc_serve_start(ctx, slots=2, max_batch=256, max_pending=1 << 20, prec=AMC_MIXED, slot_bytes=0):
    cfg = amc_serve_config(slot_bytes, slots, max_batch, max_pending, prec)
    _check(lib().amc_serve_start(ctx.handle, ctypes.byref(cfg)), "amc_serve_start")


def amc_serve_submit(ctx, opt):
    """Queue one request; returns its ticket (raises AmcError, e.g. AMC_EBUSY)."""
    t = _u64()
    _check(lib().amc_serve_submit(ctx.handle, ctypes.byref(make_option(opt)), ctypes.byref(t)), "amc_serve_submit")
    return t.value


def amc_serve_poll(ctx, ticket):
    """None while pending, else (result dict, latency seconds)."""
    r, lat = amc_result(), ctypes.c_double()
    rc = lib().amc_serve_poll(ctx.handle, ticket, ctypes.byref(r), ctypes.byref(lat))
    if rc == AMC_PENDING:
        return None
    _check(rc, "amc_serve_poll")
    return _res_dict(r), lat.value


def amc_serve_drain(ctx, cap=4096):
    """Finished requests: list of (ticket, result dict, latency seconds)."""
    tk = (_u64 * cap)()
    rs = (amc_result * cap)()
    lat = (ctypes.c_double * cap)()
    n = ctypes.c_int()
    _check(lib().amc_serve_drain(ctx.handle, tk, rs, lat, cap, ctypes.byref(n)), "amc_serve_drain")
    return [(tk[i], _res_dict(rs[i]), lat[i]) for i in range(n.value)]


def amc_serve_cancel(ctx, ticket):
    """Cancel a queued request (it then finishes with status AMC_ECANCELED);
    raises AmcError (AMC_EBUSY: already on the GPU or finished)."""
    _check(lib().amc_serve_cancel(ctx.handle, ticket), "amc_serve_cancel")


def amc_serve_stats_get(ctx):
    st = amc_serve_stats()
    _check(lib().amc_serve_stats_get(ctx.handle, ctypes.byref(st)), "amc_serve_stats_get")
    return {f: getattr(st, f) for f, _ in amc_serve_stats._fields_}


def amc_serve_stop(ctx):
    _check(lib().amc_serve_stop(ctx.handle), "amc_serve_stop")


def amc_sweep_noalloc(opt, prec, S, res, ld=None, with_greeks=False, stream=None):
    """Sweep without a context or any device allocation (scratch in a fixed
    device array of the library; see include/amc.h).  Uses the current device."""
    ld = S.shape[1] if ld is None else ld
    _check(lib().amc_sweep_noalloc(ctypes.byref(make_option(opt)), prec, _ptr(S), ld, 1 if with_greeks else 0,
                                   _ptr(res), _stream(stream)), "amc_sweep_noalloc")


def amc_sweep_noalloc_capacity():
    return lib().amc_sweep_noalloc_capacity()


def res_to_dict(res_row):
    """Device result block (AMC_RES_DOUBLES doubles, already on host) to a dict."""
    v = [float(x) for x in res_row]
    return {"price": v[0], "std_err": v[1], "delta": v[2], "vega": v[3], "degenerate_dates": int(v[4]),
            "status": int(v[5])}


# ------------------------------------------------------------ host level
def amc_price_american(ctx, S0, K, r, sigma, T, n_steps, n_paths, basis=3, type=AMC_PUT, seed=0,
                       rule=AMC_RULE_LSM, prec=AMC_MIXED):
    out = amc_result()
    _check(lib().amc_price_american(ctx.handle, S0, K, r, sigma, T, n_steps, n_paths, basis, type, seed, rule, prec,
                                    ctypes.byref(out)), "amc_price_american")
    return _res_dict(out)


def amc_price_batch(ctx, options, prec=AMC_MIXED):
    n = len(options)
    arr = (amc_option * n)(*[make_option(o) for o in options])
    out = (amc_result * n)()
    _check(lib().amc_price_batch(ctx.handle, arr, n, prec, out), "amc_price_batch")
    return [_res_dict(r) for r in out]


def amc_greeks(ctx, options, prec=AMC_MIXED):
    import numpy as np
    n = len(options)
    arr = (amc_option * n)(*[make_option(o) for o in options])
    p, d, v = (np.zeros(n) for _ in range(3))
    _check(lib().amc_greeks(ctx.handle, arr, n, prec, p.ctypes.data_as(_dp), d.ctypes.data_as(_dp),
                            v.ctypes.data_as(_dp)), "amc_greeks")
    return p, d, v


def amc_price_batch_device(ctx, options, res, prec=AMC_MIXED, stream=None):
    """Price the options on `stream` (a torch.cuda.Stream, a raw handle, or
    None for the legacy default stream) into the device tensor res (float64,
    [n, AMC_RES_DOUBLES] contiguous, input order).  Returns without waiting
    for the GPU."""
    n = len(options)
    arr = (amc_option * n)(*[make_option(o) for o in options])
    _check(lib().amc_price_batch_device(ctx.handle, arr, n, prec, _ptr(res), _stream(stream)),
           "amc_price_batch_device")


def amc_greeks_device(ctx, options, price, delta, vega, prec=AMC_MIXED, S0=None, sigma=None, res=None, stream=None):
    """Price, delta and vega of the options on `stream` into the device
    tensors price, delta, vega (float64 [n]); S0 and sigma (float64 [n]
    device tensors, optional) replace the options' spot and volatility and
    are checked on the device; res (float64 [n, AMC_RES_DOUBLES], optional)
    receives the full result blocks.  Returns without waiting for the GPU."""
    n = len(options)
    arr = (amc_option * n)(*[make_option(o) for o in options])
    _check(lib().amc_greeks_device(ctx.handle, arr, n, prec, _ptr(S0), _ptr(sigma), _ptr(price), _ptr(delta),
                                   _ptr(vega), _ptr(res), _stream(stream)), "amc_greeks_device")
