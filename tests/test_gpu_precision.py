"""The FP32-storage form against the FP64 oracle, observable by observable:
8^4 at the throughput workload's parameters (Haar start, beta 6.2, theta 1,
eps 0.005, 10 D_1 sweeps per step), after 1 and 10 steps.  The bounds are
those the DESIGN error table states (FP32 rounding of the links, ~1e-7
relative, grows by the chaotic divergence of the trajectories)."""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


BOUNDS = {1: dict(links=1e-5, plaq_re=5e-6, plaq_im=5e-6, un=2e-6, q_re=1e-4, q_im=1e-4, s_re=1e-6, s_im=1e-6),
          10: dict(links=1e-4, plaq_re=2e-5, plaq_im=2e-5, un=5e-6, q_re=1e-3, q_im=1e-3, s_re=5e-6, s_im=5e-6)}


def test_fp32_form_against_the_oracle_every_observable():
    L, beta, theta, eps, seed = (8, 8, 8, 8), 6.2, 1.0, 0.005, 1
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D1, forced_sweeps=10)
    U = O.hot_start(L, seed)
    V = 8 ** 4
    with cl.Lattice(L, beta=beta, theta=theta, prec=cl.CL_FP32_STORAGE, seed=seed, start=cl.CL_START_HOT) as lat:
        for step in range(10):
            lat.step(eps, 1)
            lat.cool(cl.make_cool(**cpar), want_report=False)
            U, _ = O.cool(L, O.cl_step(L, U, beta, theta, eps, seed, step), O.cool_params(**cpar))
            if step + 1 in BOUNDS:
                o = lat.observables()
                ref = O.observables(L, U, beta, theta)
                b = BOUNDS[step + 1]
                link_err = np.abs(lat.links() - U).max()
                print("\\nstep %d: links %.2e" % (step + 1, link_err))
                assert link_err < b["links"]
                for k in ("plaq_re", "plaq_im", "un", "q_re", "q_im", "s_re", "s_im"):
                    # extensive sums (Q, S) relative to their natural scale
                    scale = {"s_re": 6 * V * beta, "s_im": 6 * V * beta}.get(k, 1.0)
                    d = abs(o[k] - ref[k]) / scale
                    print("  %-8s oracle %+.10e  |fp32 - oracle| / scale %.2e" % (k, ref[k], d))
                    assert d < b[k], (step + 1, k, d)
