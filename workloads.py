"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds option parameters and arrival times only, and none of the
pricing arithmetic.  Both the CUDA path and the oracle receive what it
produces.  There is no public dataset for this method: every workload is drawn
from numpy's PCG64 generator with a fixed seed.

Workloads:
  single_small   one American put, S0=36, K=40, r=0.06, sigma=0.2, T=1,
                 50 dates, 2^14 paths, basis size 3, shift seed 1
  single_large   one American put, S0=100, K=100, r=0.05, sigma=0.3, T=1,
                 252 dates, 2^20 paths, basis size 4, shift seed 2
  batch_options  4096 puts/calls, seed 3: S0, K ~ U[80,120],
                 sigma ~ U[0.1,0.5], r ~ U[0,0.08], T ~ U[0.25,2],
                 n_steps ~ U{12..365}, n_paths = 2^k with k ~ U{14..18},
                 type ~ U{put, call}, basis 3, shift seed 3*2^32 + index
  serving_requests  Poisson arrivals, 2000 req/s for 60 s, seed 4, option
                 parameters drawn as in batch_options
  greeks_options 1024 puts, seed 5, drawn as batch_options but with
                 2^18 paths and 100 dates
  fig1_options   the Longstaff-Schwartz Table 1 put for m = 1..16, then
                 every 8th m to 360 and m = 365 exercise dates, one shift
                 seed, for LSM and the paper's rule
A basis of size p spans {1, S, .., S^(p-1)}; the library and the oracle
regress on powers of the moneyness y = S/K - 1, the same span.
"""
from dataclasses import asdict, dataclass

import numpy as np

PUT, CALL = 0, 1
RULE_LSM, RULE_PAPER_UB, RULE_EUROPEAN = 0, 1, 2


@dataclass
class Option:
    S0: float
    K: float
    r: float
    sigma: float
    T: float
    n_steps: int
    n_paths: int
    basis: int = 3
    type: int = PUT
    seed: int = 0
    rule: int = RULE_LSM

    def as_dict(self):
        return asdict(self)

    @property
    def path_steps(self):
        return self.n_paths * self.n_steps


def single_small():
    return Option(36.0, 40.0, 0.06, 0.2, 1.0, 50, 2 ** 14, basis=3, type=PUT, seed=1)


def single_large():
    return Option(100.0, 100.0, 0.05, 0.3, 1.0, 252, 2 ** 20, basis=4, type=PUT, seed=2)


def _draw(rng, n, seed_base, n_paths=None, n_steps=None, type_=None, basis=3):
    S0 = rng.uniform(80, 120, n)
    K = rng.uniform(80, 120, n)
    sigma = rng.uniform(0.1, 0.5, n)
    r = rng.uniform(0.0, 0.08, n)
    T = rng.uniform(0.25, 2.0, n)
    m = rng.integers(12, 366, n)
    k = rng.integers(14, 19, n)
    tp = rng.integers(0, 2, n)
    out = []
    for i in range(n):
        out.append(Option(float(S0[i]), float(K[i]), float(r[i]), float(sigma[i]), float(T[i]),
                          int(m[i]) if n_steps is None else n_steps,
                          int(2 ** int(k[i])) if n_paths is None else n_paths,
                          basis=basis, type=int(tp[i]) if type_ is None else type_,
                          seed=seed_base + i))
    return out


def batch_options(n=4096, seed=3):
    """The 4096-option batch (parameters drawn vectorised, in the order listed above)."""
    return _draw(np.random.default_rng(seed), n, seed * 2 ** 32)


def greeks_options(n=1024, seed=5):
    return _draw(np.random.default_rng(seed), n, seed * 2 ** 32, n_paths=2 ** 18, n_steps=100, type_=PUT)


def serving_requests(rate=2000.0, duration=60.0, seed=4):
    """(arrival_times_s, options): exponential gaps at `rate` per second."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, int(rate * duration * 1.5) + 100)
    t = np.cumsum(gaps)
    t = t[t < duration]
    return t, _draw(rng, len(t), seed * 2 ** 32)


def scaled(opt, n_paths=None, n_steps=None):
    """Same option with another path or date count (test sizes)."""
    d = opt.as_dict()
    if n_paths is not None:
        d["n_paths"] = n_paths
    if n_steps is not None:
        d["n_steps"] = n_steps
    return Option(**d)


# Fig. 1 grid: every m in 1..16, then every 8th m up to 360, and m = 365
FIG1_DATES = tuple(range(1, 17)) + tuple(range(24, 361, 8)) + (365,)
# the nested power-of-two grids within it (each contains the coarser ones)
FIG1_NESTED = (1, 2, 4, 8, 16, 32, 64, 128, 256)


def fig1_options(dates=FIG1_DATES, n_paths=2 ** 16, seed=21, rules=(RULE_LSM, RULE_PAPER_UB)):
    """Value vs number of exercise dates (the paper's Fig. 1, which prints no
    parameters): the Longstaff-Schwartz Table 1 put (S0 36, K 40, r 6 %,
    sigma 20 %, T 1 year, basis 3) on the same shift seed for every m from
    1 to 365 (FIG1_DATES); its power-of-two date grids (FIG1_NESTED) are
    nested.  Ordered rule-major, then by m."""
    return [Option(36.0, 40.0, 0.06, 0.2, 1.0, m, n_paths, basis=3, type=PUT, seed=seed, rule=rule)
            for rule in rules for m in dates]
