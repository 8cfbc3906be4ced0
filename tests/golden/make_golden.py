"""Write the stored expected values under tests/golden/ by calling only the oracle.

cfg0_trajectory.json: SU(3) Wilson action on a 4^4 periodic lattice, beta = 6,
theta = 0; cold start followed by the random SL(3,C) gauge transformation
Omega_x = exp(i w_a lambda_a), w_a = i N(0, 0.05) (seed 1); 20 CL steps at
eps = 0.01 with Philox noise from seed 1, each followed by 5 cooling sweeps at
alpha_gf = 1 (D_0, fixed count); plaquette and unitarity norm after every step.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

CFG0 = dict(L=[4, 4, 4, 4], beta=6.0, theta=0.0, seed=1, sigma=0.05, eps=0.01, n_steps=20,
            sweeps=5, alpha=1.0)


def cfg0():
    c = CFG0
    L = tuple(c["L"])
    U = O.random_gauge(L, O.cold_start(L), c["seed"], c["sigma"])
    start = O.observables(L, U, c["beta"], c["theta"])
    cp = O.cool_params(c["eps"], c["alpha"], O.D0, forced_sweeps=c["sweeps"])
    U, recs = O.trajectory(L, U, c["beta"], c["theta"], c["eps"], c["seed"], 0, c["n_steps"], cp, 1)
    return {"config": c, "start": start, "steps": recs}


if __name__ == "__main__":
    out = os.path.join(HERE, "cfg0_trajectory.json")
    with open(out, "w") as fh:
        json.dump(cfg0(), fh, indent=1)
    print("wrote", out)
