"""Seeded synthetic workloads: chain ensembles and request traces.

Only parameter draws live here (lattice extents, couplings, seeds, arrival
times); none of the method's arithmetic.  Both the benchmark and the tests
take their inputs from these recipes.

* ensemble(n): independent chains with L in {8, 12, 16} (uniform), beta
  uniform in [5.6, 6.2], theta uniform over {0, 0.5, 1, 1.5, 2}.
* trace(n, rate): requests arriving as a Poisson process of the given rate
  (exponential gaps), L = round(exp(U[ln 4, ln 24])), beta ~ U[5.6, 6.2],
  theta ~ U[0, 2], steps ~ U{100, ..., 2000}.
Every chain gets its own Philox seed, so its noise does not depend on what
else runs beside it.
"""
import math

import numpy as np

ENSEMBLE_SIZES = (8, 12, 16)
ENSEMBLE_THETAS = (0.0, 0.5, 1.0, 1.5, 2.0)
BETA_RANGE = (5.6, 6.2)
TRACE_L_RANGE = (4, 24)
TRACE_STEPS = (100, 2000)


def ensemble(n=64, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        L = int(rng.choice(ENSEMBLE_SIZES))
        out.append(dict(L=(L, L, L, L), beta=float(rng.uniform(*BETA_RANGE)),
                        theta=float(rng.choice(ENSEMBLE_THETAS)), seed=1000 + i))
    return out


def trace(n=200, rate=20.0, seed=0, steps=TRACE_STEPS, l_range=TRACE_L_RANGE):
    """Requests sorted by arrival time t (seconds from the first draw)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    lo, hi = math.log(l_range[0]), math.log(l_range[1])
    for i in range(n):
        t += float(rng.exponential(1.0 / rate))
        L = int(round(math.exp(rng.uniform(lo, hi))))
        out.append(dict(id=i, t=t, L=(L, L, L, L), beta=float(rng.uniform(*BETA_RANGE)),
                        theta=float(rng.uniform(0.0, 2.0)),
                        steps=int(rng.integers(steps[0], steps[1] + 1)), seed=5000 + i))
    return out


def sites(chain):
    L = chain["L"]
    return L[0] * L[1] * L[2] * L[3]
