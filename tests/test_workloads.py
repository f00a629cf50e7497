"""The seeded input recipes: every generated workload has the shapes, ranges
and seeds its documentation states, and draws the same options on every call
(CPU)."""
import numpy as np
import pytest

import workloads


def _fields(opts):
    return {k: np.array([getattr(o, k) for o in opts]) for k in
            ("S0", "K", "r", "sigma", "T", "n_steps", "n_paths", "basis", "type", "seed", "rule")}


def test_single_options():
    s, b = workloads.single_small(), workloads.single_large()
    assert (s.S0, s.K, s.r, s.sigma, s.T, s.n_steps, s.n_paths, s.basis, s.type, s.seed) == \
        (36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, 3, workloads.PUT, 1)
    assert (b.S0, b.K, b.r, b.sigma, b.T, b.n_steps, b.n_paths, b.basis, b.type, b.seed) == \
        (100.0, 100.0, 0.05, 0.3, 1.0, 252, 2 ** 20, 4, workloads.PUT, 2)
    assert s.rule == b.rule == workloads.RULE_LSM
    assert b.path_steps == 252 * 2 ** 20


def test_batch_recipe():
    opts = workloads.batch_options()
    f = _fields(opts)
    assert len(opts) == 4096
    for k, lo, hi in (("S0", 80, 120), ("K", 80, 120), ("sigma", 0.1, 0.5), ("r", 0.0, 0.08), ("T", 0.25, 2.0)):
        assert f[k].min() >= lo and f[k].max() < hi, k
    assert f["n_steps"].min() >= 12 and f["n_steps"].max() <= 365
    assert set(np.log2(f["n_paths"]).astype(int).tolist()) <= set(range(14, 19))
    assert (2 ** np.log2(f["n_paths"]).astype(int) == f["n_paths"]).all()
    assert set(f["type"].tolist()) == {workloads.PUT, workloads.CALL}
    assert (f["basis"] == 3).all() and (f["rule"] == workloads.RULE_LSM).all()
    assert (f["seed"] == 3 * 2 ** 32 + np.arange(4096)).all()
    # E[N] = (2^14 + .. + 2^18) / 5 = 101 580.8, E[m] = 188.5: the sample sits within a few standard errors
    assert abs(f["n_paths"].mean() - 101580.8) < 4 * f["n_paths"].std() / np.sqrt(4096)
    assert abs(f["n_steps"].mean() - 188.5) < 4 * f["n_steps"].std() / np.sqrt(4096)
    total = float((f["n_paths"] * f["n_steps"]).sum())
    assert 7.4e10 < total < 8.4e10                      # about 7.8e10 path-steps in all
    # drawn vectorised, one field after another, from default_rng(3)
    rng = np.random.default_rng(3)
    assert np.array_equal(f["S0"], rng.uniform(80, 120, 4096))
    assert np.array_equal(f["K"], rng.uniform(80, 120, 4096))


def test_batch_is_reproducible():
    a, b = workloads.batch_options(), workloads.batch_options()
    assert [o.as_dict() for o in a] == [o.as_dict() for o in b]


def test_greeks_recipe():
    opts = workloads.greeks_options()
    f = _fields(opts)
    assert len(opts) == 1024
    assert (f["type"] == workloads.PUT).all() and (f["n_paths"] == 2 ** 18).all() and (f["n_steps"] == 100).all()
    assert (f["seed"] == 5 * 2 ** 32 + np.arange(1024)).all()
    assert f["S0"].min() >= 80 and f["S0"].max() < 120 and f["sigma"].min() >= 0.1 and f["sigma"].max() < 0.5


def test_serving_arrivals():
    t, opts = workloads.serving_requests()
    assert len(t) == len(opts)
    assert (np.diff(t) > 0).all() and t[0] > 0 and t[-1] < 60.0
    # Poisson at 2000/s over 60 s: about 120 000 requests, exponential gaps of mean 0.5 ms
    assert abs(len(t) - 120000) < 4 * np.sqrt(120000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 5e-4) < 4 * 5e-4 / np.sqrt(len(gaps))
    assert abs(np.median(gaps) / gaps.mean() - np.log(2)) < 0.02          # exponential: median = mean ln 2
    f = _fields(opts[:4096])
    assert f["n_steps"].min() >= 12 and f["n_steps"].max() <= 365
    assert (f["seed"] == 4 * 2 ** 32 + np.arange(4096)).all()
    t2, _ = workloads.serving_requests(duration=1.0)
    assert np.array_equal(t2, t[t < 1.0])                                # a shorter replay is a prefix


@pytest.mark.parametrize("n_paths,n_steps", [(5, None), (None, 7), (123, 512)])
def test_scaled_keeps_the_rest(n_paths, n_steps):
    o = workloads.single_large()
    s = workloads.scaled(o, n_paths=n_paths, n_steps=n_steps)
    d, e = o.as_dict(), s.as_dict()
    assert e["n_paths"] == (n_paths or d["n_paths"]) and e["n_steps"] == (n_steps or d["n_steps"])
    for k in d:
        if k not in ("n_paths", "n_steps"):
            assert d[k] == e[k]


def test_fig1_grid_spans_1_to_365_on_one_shift():
    opts = workloads.fig1_options()
    assert len(opts) == 2 * len(workloads.FIG1_DATES)
    lsm = [o for o in opts if o.rule == workloads.RULE_LSM]
    assert [o.n_steps for o in lsm] == list(workloads.FIG1_DATES)
    assert set(range(1, 17)) <= set(workloads.FIG1_DATES) and workloads.FIG1_DATES[-1] == 365
    assert all(b - a <= 8 for a, b in zip(workloads.FIG1_DATES, workloads.FIG1_DATES[1:]))
    assert set(workloads.FIG1_NESTED) <= set(workloads.FIG1_DATES)
    for a, b in zip(workloads.FIG1_NESTED, workloads.FIG1_NESTED[1:]):
        assert b % a == 0                                                 # every grid contains the coarser one
    assert len({(o.S0, o.K, o.r, o.sigma, o.T, o.seed, o.n_paths) for o in opts}) == 1
