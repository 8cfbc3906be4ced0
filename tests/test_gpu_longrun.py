"""Long-run agreement in distribution.

Complex-Langevin trajectories decorrelate chaotically, so after many steps
two arithmetic forms (or the GPU and the oracle) can only agree
statistically.  Here independent ensembles -- disjoint Philox seeds, cold
starts, CL with the adaptive step size (k_ref 12) and adaptive cooling
(alpha_ad = 0.1 / D_2, 0..10 sweeps) --
are run long enough to thermalise, and the ensemble means of Re/Im of the
plaquette, the unitarity norm and Re/Im Q_L (first 20 % of each chain
dropped, errors from the chain-to-chain scatter) must agree within 4
standard errors: the FP32-storage and DF64 forms against FP64 on 8^4, and
the FP64 kernels against the FP64 oracle on 4^4.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl, studies

pytestmark = pytest.mark.gpu

Z_MAX = 4.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


@pytest.mark.parametrize("theta", [0.5, 2.0])
def test_forms_agree_in_distribution(theta):
    L, beta, steps, k = (8, 8, 8, 8), 6.0, 600, 6
    st = {}
    for name, prec, off in (("fp64", cl.CL_FP64, 0), ("fp32", cl.CL_FP32_STORAGE, 100), ("df64", cl.CL_DF64, 200)):
        ser = studies.longrun(L, beta, theta, prec, [300 + off + i for i in range(k)], steps, k_ref=12.0)
        st[name] = studies.chain_means(ser)
        assert st[name]["dropped"] == 0
    for name, floor in (("fp32", 1e-6), ("df64", 1e-12)):
        z = studies.compare_means(st[name], st["fp64"], floor)
        assert np.all(z < Z_MAX), (name, dict(zip(studies.SERIES_KEYS, z)))
    # the runs are long enough to leave the cold start: the plaquette has relaxed
    assert st["fp64"]["mean"][0] < 0.8


def test_gpu_matches_oracle_in_distribution():
    L, beta, theta, eps, steps, every, k = (4, 4, 4, 4), 6.0, 1.0, 0.005, 600, 10, 4
    gpu = studies.longrun(L, beta, theta, cl.CL_FP64, [500 + i for i in range(k)], steps, every=every, eps=eps)
    cp = studies.longrun_cool(eps)
    ocp = O.cool_params(cp.eps, cp.alpha, O.D2_MEANABS, cp.n_min, cp.n_max, cp.tol_rel, cp.d_floor, cp.d_guard)
    orc = np.zeros_like(gpu)
    for i in range(k):
        _, rec = O.trajectory(L, O.cold_start(L), beta, theta, eps, 600 + i, 0, steps, ocp, every)
        orc[i] = [[r[key] for key in studies.SERIES_KEYS] for r in rec]
    a, b = studies.chain_means(gpu), studies.chain_means(orc)
    z = studies.compare_means(a, b)
    assert np.all(z < Z_MAX), dict(zip(studies.SERIES_KEYS, z))
