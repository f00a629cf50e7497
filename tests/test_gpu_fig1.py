"""Value vs number of exercise dates (the paper's Fig. 1) on the GPU: every
(dates, rule) point vs the FP64 oracle on identical points, |dP| <= 2e-4 K and
equal degenerate-date counts, through the batch call; and the curve's shape
(LSM non-decreasing on nested grids, the paper's rule above it)."""
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1205_0106_gb300 as amc
    return amc


@pytest.fixture(scope="module")
def ctx(amc):
    c = amc.Context(0, arena_bytes=8 << 30)
    yield c
    c.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_fig1_points_vs_oracle(amc, ctx, prec):
    opts = workloads.fig1_options(n_paths=2 ** 14)
    res = amc.amc_price_batch(ctx, opts, prec)
    for o, r in zip(opts, res):
        ref = oracle.price(o.S0, o.K, o.r, o.sigma, o.T, o.n_steps, o.n_paths, basis=o.basis, type=o.type,
                           seed=o.seed, rule=o.rule)
        assert r["status"] == 0
        assert abs(r["price"] - ref["price"]) <= 2e-4 * o.K, (o, r, ref)
        assert r["degenerate_dates"] == ref["degenerate_dates"]


def test_fig1_curve_shape(amc, ctx):
    opts = workloads.fig1_options()
    res = amc.amc_price_batch(ctx, opts, amc.AMC_MIXED)
    n = len(workloads.FIG1_DATES)
    lsm, ub = res[:n], res[n:]
    for a, b in zip(lsm, lsm[1:]):
        assert b["price"] >= a["price"] - 3 * (a["std_err"] + b["std_err"])
    for l, u in zip(lsm, ub):
        assert u["price"] >= l["price"] - 3 * l["std_err"]
    assert lsm[-1]["price"] - lsm[0]["price"] > 0.5
