"""The allocation-free sweep entry point (amc_sweep_noalloc) against the
context-based one (amc_sweep) on the same paths.

amc_sweep_noalloc serves callers that may not allocate device memory (a
framework that owns the device-memory budget, a latency-critical loop that
cannot take cudaMalloc's device-wide synchronisation, a hook without an
amc_ctx).  It runs the same kernels with the same launch plan as amc_sweep,
with its scratch in a fixed device array inside the library, so its results
must equal amc_sweep's bit for bit.  The array keeps the previous call's
contents, and one region of it holds the FP64 and pathwise sweeps' double
partial sums as well as the mixed sweep's tagged exchange units, so the
tests call it twice in a row on each case and also alternate the kinds of
sweep: no call may see leftovers of an earlier one.  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    ctx = amc.Context(0, arena_bytes=1 << 30)
    yield amc, ctx, torch
    ctx.close()


CASES = [
    ("lsm_mixed", workloads.single_small(), 1),
    ("lsm_fp64", workloads.single_small(), 0),
    ("lsm_large_group", workloads.scaled(workloads.single_large(), n_paths=2 ** 18 + 5, n_steps=100), 1),
    ("paper_rule", workloads.Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 3000, seed=3, rule=1), 1),
    ("european_call", workloads.Option(110.0, 100.0, 0.03, 0.3, 0.5, 12, 5000, type=1, seed=4, rule=2), 0),
    ("lsm_fp64_wide", workloads.scaled(workloads.single_large(), n_paths=2 ** 17, n_steps=120), 0),
]
BY_NAME = {c[0]: c for c in CASES}


def _paths_and_reference(amc, ctx, torch, opt, prec):
    """Paths of opt in precision prec and amc_sweep's result block on them."""
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.empty((opt.n_steps, amc.amc_path_ld(opt.n_paths)), dtype=dt, device="cuda")
    amc.amc_generate_paths(ctx, opt, prec, S)
    ref = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_sweep(ctx, opt, prec, S, ref)
    torch.cuda.synchronize()
    want = ref.cpu()[:6]            # price, std_err, delta, vega, degenerate dates, status
    assert amc.res_to_dict(ref.cpu().numpy())["status"] == 0
    return S, want


def _noalloc(amc, torch, opt, prec, S):
    got = torch.full((amc.AMC_RES_DOUBLES,), float("nan"), dtype=torch.float64, device="cuda")
    amc.amc_sweep_noalloc(opt, prec, S, got)
    torch.cuda.synchronize()
    return got.cpu()[:6]


@pytest.mark.parametrize("name,opt,prec", CASES, ids=[c[0] for c in CASES])
def test_noalloc_sweep_equals_context_sweep_on_two_calls(env, name, opt, prec):
    amc, ctx, torch = env
    S, want = _paths_and_reference(amc, ctx, torch, opt, prec)
    for call in range(2):
        got = _noalloc(amc, torch, opt, prec, S)
        assert torch.equal(got, want), (call, got, want)


def test_noalloc_alternating_kinds_leave_nothing_behind(env):
    """Mixed LSM calls after FP64 LSM and pathwise calls (whose double partial
    sums occupy the bytes the mixed sweep's exchange units use) and the other
    way round, twice over: every result equals amc_sweep's bit for bit."""
    amc, ctx, torch = env
    order = ["lsm_fp64_wide", "lsm_large_group", "paper_rule", "lsm_mixed", "lsm_fp64", "lsm_large_group",
             "european_call", "lsm_large_group"]
    data = {}
    for name in set(order):
        _, opt, prec = BY_NAME[name]
        data[name] = _paths_and_reference(amc, ctx, torch, opt, prec)
    for rnd in range(2):
        for name in order:
            _, opt, prec = BY_NAME[name]
            S, want = data[name]
            got = _noalloc(amc, torch, opt, prec, S)
            assert torch.equal(got, want), (rnd, name, got, want)


def test_noalloc_rejects_options_beyond_its_scratch(env):
    """An FP64 LSM option with 512 dates and 2^20 paths needs more scratch
    than the array holds: AMC_EINVAL before any device work.  The path array
    has the option's full shape, so even a call that wrongly went ahead would
    read only memory it owns."""
    amc, ctx, torch = env
    big = workloads.scaled(workloads.single_large(), n_steps=512)
    S = torch.empty((big.n_steps, amc.amc_path_ld(big.n_paths)), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_sweep_noalloc(big, amc.AMC_FP64, S, res)
    assert ei.value.code == amc.AMC_EINVAL
    assert amc.amc_sweep_noalloc_capacity() == 16 << 20
    torch.cuda.synchronize()
    assert torch.count_nonzero(res).item() == 0


def test_noalloc_rejects_options_beyond_the_register_resident_sweep(env):
    """amc_sweep takes a mixed LSM option one path above the register-resident
    sweep's limit to the streaming sweep; amc_sweep_noalloc has no fallback
    and returns AMC_EINVAL before any device work (full-shape paths again)."""
    amc, ctx, torch = env
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    limit = min(sms, 160) * 7680
    assert amc.amc_plan_sweep(limit, sms)[0] == min(sms, 160)
    opt = workloads.scaled(workloads.single_small(), n_paths=limit + 1, n_steps=2)
    S = torch.empty((opt.n_steps, amc.amc_path_ld(opt.n_paths)), dtype=torch.float32, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_sweep_noalloc(opt, amc.AMC_MIXED, S, res)
    assert ei.value.code == amc.AMC_EINVAL
    torch.cuda.synchronize()
    assert torch.count_nonzero(res).item() == 0
