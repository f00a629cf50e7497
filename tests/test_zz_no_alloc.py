"""The allocation-free sweep entry point (amc_sweep_noalloc) against the
context-based one (amc_sweep) on the same paths.

amc_sweep_noalloc serves callers that may not allocate device memory (a
framework that owns the device-memory budget, a latency-critical loop that
cannot take cudaMalloc's device-wide synchronisation, a hook without an
amc_ctx).  Its scratch is a fixed device array inside the library that
keeps the previous call's contents, so the test calls it twice in a row on
each case: the second call must not see leftovers of the first.  This file
is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
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
]


@pytest.mark.parametrize("name,opt,prec", CASES, ids=[c[0] for c in CASES])
def test_noalloc_sweep_matches_context_sweep_on_two_calls(env, name, opt, prec):
    amc, ctx, torch = env
    dt = torch.float64 if prec == amc.AMC_FP64 else torch.float32
    S = torch.empty((opt.n_steps, amc.amc_path_ld(opt.n_paths)), dtype=dt, device="cuda")
    amc.amc_generate_paths(ctx, opt, prec, S)
    ref = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    amc.amc_sweep(ctx, opt, prec, S, ref)
    torch.cuda.synchronize()
    want = amc.res_to_dict(ref.cpu().numpy())
    assert want["status"] == 0
    for call in range(2):
        got_t = torch.full((amc.AMC_RES_DOUBLES,), float("nan"), dtype=torch.float64, device="cuda")
        amc.amc_sweep_noalloc(opt, prec, S, got_t)
        torch.cuda.synchronize()
        got = amc.res_to_dict(got_t.cpu().numpy())
        assert got["status"] == 0, (call, got)
        assert abs(got["price"] - want["price"]) <= 2e-4 * opt.K, (call, got, want)
        assert abs(got["std_err"] - want["std_err"]) <= 2e-4 * opt.K, (call, got, want)
        assert got["degenerate_dates"] == want["degenerate_dates"], (call, got, want)


def test_noalloc_rejects_options_beyond_its_scratch(env):
    amc, ctx, torch = env
    big = workloads.scaled(workloads.single_large(), n_steps=512)
    S = torch.empty((1, amc.amc_path_ld(big.n_paths)), dtype=torch.float64, device="cuda")
    res = torch.zeros(amc.AMC_RES_DOUBLES, dtype=torch.float64, device="cuda")
    with pytest.raises(amc.AmcError) as ei:
        amc.amc_sweep_noalloc(big, amc.AMC_FP64, S, res)
    assert ei.value.code == amc.AMC_EINVAL
    assert amc.amc_sweep_noalloc_capacity() == 16 << 20
