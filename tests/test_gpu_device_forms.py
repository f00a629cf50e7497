"""The stream and device-output forms of the batched and Greeks calls
(amc_price_batch_device, amc_greeks_device) through the C ABI, on a torch
side stream: results bit-identical to the blocking host forms, ordered on the
caller's stream, spot and volatility read from device tensors and checked on
the device, and the context's next calls ordered after them."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    # a small arena: the batch below takes several waves on both batch streams
    ctx = amc.Context(0, arena_bytes=320 << 20)
    yield amc, ctx, torch
    ctx.close()


def _opts(n, n_paths_max=2 ** 15):
    return [workloads.scaled(o, n_paths=min(o.n_paths, n_paths_max)) for o in workloads.batch_options(n=n)]


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "fp64"])
def test_batch_device_form_equals_host_form(env, prec):
    amc, ctx, torch = env
    opts = _opts(40 if prec == 1 else 12)
    host = amc.amc_price_batch(ctx, opts, prec)
    st = torch.cuda.Stream()
    res = torch.full((len(opts), amc.AMC_RES_DOUBLES), float("nan"), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(st):
        res.fill_(-7.0)                                  # queued on st before the call: must be overwritten
        amc.amc_price_batch_device(ctx, opts, res, prec, stream=st)
        got = res.cpu()                                  # on st: ordered after the library's work
    st.synchronize()
    for i, h in enumerate(host):
        d = amc.res_to_dict(got[i].numpy())
        assert d["status"] == 0 and h["status"] == 0
        assert d["price"] == h["price"] and d["std_err"] == h["std_err"], (i, d, h)
        assert d["degenerate_dates"] == h["degenerate_dates"]


def test_greeks_device_form_with_device_spot_and_volatility(env):
    amc, ctx, torch = env
    base = [workloads.Option(**{**o.as_dict(), "type": workloads.PUT}) for o in _opts(10, 2 ** 14)]
    rng = np.random.default_rng(5)
    S0 = rng.uniform(80, 120, len(base))
    sig = rng.uniform(0.1, 0.5, len(base))
    want = [workloads.Option(**{**o.as_dict(), "S0": float(a), "sigma": float(b)}) for o, a, b in zip(base, S0, sig)]
    hp, hd, hv = amc.amc_greeks(ctx, want, amc.AMC_MIXED)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s0 = torch.tensor(S0, dtype=torch.float64, device="cuda")
        sg = torch.tensor(sig, dtype=torch.float64, device="cuda")
        p, d, v = (torch.empty(len(base), dtype=torch.float64, device="cuda") for _ in range(3))
        res = torch.empty((len(base), amc.AMC_RES_DOUBLES), dtype=torch.float64, device="cuda")
        # the options' own S0 and sigma are placeholders: the device tensors replace them
        amc.amc_greeks_device(ctx, base, p, d, v, amc.AMC_MIXED, S0=s0, sigma=sg, res=res, stream=st)
        out = [t.cpu().numpy() for t in (p, d, v, res)]
    st.synchronize()
    assert np.array_equal(out[0], hp) and np.array_equal(out[1], hd) and np.array_equal(out[2], hv)
    assert all(amc.res_to_dict(r)["status"] == 0 for r in out[3])


def test_greeks_device_form_rejects_bad_device_inputs_per_option(env):
    amc, ctx, torch = env
    base = [workloads.Option(**{**o.as_dict(), "type": workloads.PUT}) for o in _opts(6, 2 ** 14)]
    S0 = np.array([o.S0 for o in base])
    sig = np.array([o.sigma for o in base])
    S0[1] = -5.0
    sig[3] = float("nan")
    S0[4] = float("inf")
    s0 = torch.tensor(S0, dtype=torch.float64, device="cuda")
    sg = torch.tensor(sig, dtype=torch.float64, device="cuda")
    p, d, v = (torch.empty(len(base), dtype=torch.float64, device="cuda") for _ in range(3))
    res = torch.empty((len(base), amc.AMC_RES_DOUBLES), dtype=torch.float64, device="cuda")
    amc.amc_greeks_device(ctx, base, p, d, v, amc.AMC_MIXED, S0=s0, sigma=sg, res=res,
                          stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    good = [0, 2, 5]
    hp, hd, hv = amc.amc_greeks(ctx, [base[i] for i in good], amc.AMC_MIXED)
    pc, dc, vc, rc = p.cpu().numpy(), d.cpu().numpy(), v.cpu().numpy(), res.cpu().numpy()
    for k, i in enumerate(good):
        assert pc[i] == hp[k] and dc[i] == hd[k] and vc[i] == hv[k]
        assert amc.res_to_dict(rc[i])["status"] == 0
    for i in (1, 3, 4):
        assert math.isnan(pc[i]) and math.isnan(dc[i]) and math.isnan(vc[i])
        assert amc.res_to_dict(rc[i])["status"] == amc.AMC_EINVAL


def test_device_form_validates_on_the_host_before_device_work(env):
    amc, ctx, torch = env
    res = torch.zeros((2, amc.AMC_RES_DOUBLES), dtype=torch.float64, device="cuda")
    bad = [workloads.single_small(), workloads.scaled(workloads.single_small(), n_steps=0)]
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_price_batch_device(ctx, bad, res)
    assert ei.value.code == amc.AMC_EINVAL
    paper = [workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 5, 100, rule=1)]
    p, d, v = (torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(3))
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_greeks_device(ctx, paper, p, d, v)
    assert ei.value.code == amc.AMC_EINVAL
    torch.cuda.synchronize()
    assert torch.count_nonzero(res).item() == 0


def test_context_calls_after_a_device_batch_are_ordered_after_it(env):
    """A blocking single-option call right after an asynchronous device batch
    reuses the arena the batch's waves use: it must wait for them on the
    GPU, and both results must be right."""
    amc, ctx, torch = env
    opts = _opts(30)
    host = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED)
    o = workloads.single_small()
    alone = amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                   o.rule, amc.AMC_MIXED)
    st = torch.cuda.Stream()
    res = torch.empty((len(opts), amc.AMC_RES_DOUBLES), dtype=torch.float64, device="cuda")
    amc.amc_price_batch_device(ctx, opts, res, amc.AMC_MIXED, stream=st)
    again = amc.amc_price_american(ctx, o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, o.basis, o.type, o.seed,
                                   o.rule, amc.AMC_MIXED)
    st.synchronize()
    assert again["price"] == alone["price"]
    got = res.cpu().numpy()
    for i, h in enumerate(host):
        assert got[i][0] == h["price"], (i, got[i], h)


def test_profiling_counts_every_launch_and_its_path_steps(env):
    """Opt-in device timing: a batch's path-generation and sweep launches are
    timed and their path-steps add up to the batch's; off again, nothing is
    recorded."""
    amc, ctx, torch = env
    opts = _opts(20)
    ctx.profile()                                        # clear
    ctx.set_profiling(True)
    res = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED)
    prof = ctx.profile()
    ctx.set_profiling(False)
    steps = sum(o.n_paths * o.n_steps for o in opts)
    assert all(r["status"] == 0 for r in res)
    assert prof["gen_path_steps"] == steps and prof["sweep_path_steps"] == steps
    assert prof["gen_launches"] >= 1 and prof["sweep_launches"] == prof["gen_launches"]
    assert prof["gen_ms"] > 0.0 and prof["sweep_ms"] > 0.0
    amc.amc_price_batch(ctx, opts, amc.AMC_MIXED)
    assert ctx.profile()["sweep_launches"] == 0
