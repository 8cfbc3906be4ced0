"""The SU(2) Polyakov-chain kernel (one CTA per chain, a whole chunk of
steps per launch) against the chain oracle, and the exact answer
<(1/2) Tr(U_1 ... U_N)> = I_2(beta) / I_1(beta) from an ensemble of chains."""
import numpy as np
import pytest
import scipy.special

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


ADAPT = dict(alpha=1.0, mode=cl.CL_D2_MEANABS, n_min=1, n_max=8, tol_rel=0.02)


@pytest.mark.parametrize("n", [1, 5, 33, 100])
def test_chains_against_the_oracle(n):
    betas = [1.5, 1.0 + 0.5j, 0.5 - 0.25j, 1.0 - 0.3j]
    seeds = [11, 12, 13, 14]
    eps, steps, sigma = 0.01, 10, 0.1
    cp = cl.make_cool(eps, **ADAPT)
    with cl.PolyakovChains(len(betas), n, betas, seeds, gauge_sigma=sigma) as pc:
        start = pc.links()
        rec = pc.run(steps, eps, cp, obs_every=1)
        end = pc.links()
        assert pc.step_count == steps
    ocp = O.cool_params(eps, **ADAPT)
    for c, (b, sd) in enumerate(zip(betas, seeds)):
        U0 = O.pc_random_gauge(O.pc_cold(n), sd, sigma)
        assert np.abs(start[c] - U0).max() < 1e-14
        U, orec = O.pc_trajectory(U0, b, eps, sd, 0, steps, ocp)
        assert np.array_equal(rec[:, c, 4], orec[:, 4]), c  # sweep counts
        assert np.abs(rec[:, c, :3] - orec[:, :3]).max() < 1e-11, c
        assert np.abs(end[c] - U).max() < 1e-11, c


@pytest.mark.parametrize("n,mode", [(600, cl.CL_D2_MEANABS), (1000, cl.CL_D1), (1000, cl.CL_D0)])
def test_long_chains_cooling_only(n, mode):
    """Sec. 4's experiment: a gauge-transformed unitary chain cooled with no
    Langevin update (eps = 0), one sweep per record; the unitarity norm after
    every sweep against the oracle (long products of CL-updated SL(2,C) links
    overflow at these lengths, so the CL part is exercised on shorter chains)."""
    cp = cl.make_cool(0.01, 1.0, mode, forced_sweeps=1)
    with cl.PolyakovChains(2, n, [1.0, 1.0 + 0.5j], [3, 4], gauge_sigma=0.1) as pc:
        rec = pc.run(20, 0.0, cp, obs_every=1)
        U = pc.links()
    ocp = O.cool_params(0.01, 1.0, mode, forced_sweeps=1)
    for c, sd in enumerate([3, 4]):
        U0 = O.pc_random_gauge(O.pc_cold(n), sd, 0.1)
        Uo, orec = O.pc_trajectory(U0, [1.0, 1.0 + 0.5j][c], 0.0, sd, 0, 20, ocp)
        assert np.abs(rec[:, c, 2] - orec[:, 2]).max() < 1e-12
        assert np.abs(U[c] - Uo).max() < 1e-11
        if mode != cl.CL_D2_MEANABS:  # D_0, D_1: the distance decreases sweep by sweep
            assert np.all(np.diff(rec[:, c, 2]) < 0)
        else:  # D_2's normalised step reaches a plateau instead
            assert rec[-1, c, 2] < rec[0, c, 2] - 0.05


def test_chunks_and_no_cooling():
    """Runs split over several calls and launches (256 steps each) equal one
    oracle trajectory; without cooling too."""
    n, b, sd, eps = 7, 1.2 + 0.3j, 5, 0.005
    with cl.PolyakovChains(1, n, b, [sd], gauge_sigma=0.05) as pc:
        pc.run(300, eps, None, obs_every=0)
        rec = pc.run(20, eps, None, obs_every=5)
        U = pc.links()[0]
    U0 = O.pc_random_gauge(O.pc_cold(n), sd, 0.05)
    Uo, orec = O.pc_trajectory(U0, b, eps, sd, 0, 320)
    assert np.abs(U - Uo).max() < 1e-10
    assert np.abs(rec[:, 0, :3] - orec[304::5, :3]).max() < 1e-10


@pytest.mark.parametrize("beta", [1.5, 1.0 + 0.5j])
def test_exact_answer_from_an_ensemble(beta):
    """512 independent 4-link chains, 3000 steps at eps = 0.005 with adaptive
    D_2 cooling: the mean of (1/2) Tr(U_1..U_4) over chains and the last 2000
    steps within 5 standard errors (chains are independent) plus 0.01 for the
    O(eps) bias of the Euler step."""
    exact = scipy.special.iv(2, beta) / scipy.special.iv(1, beta)
    n_chains = 512
    cp = cl.make_cool(0.01, 1.0, cl.CL_D2_MEANABS, n_min=1, n_max=10, tol_rel=0.01)
    with cl.PolyakovChains(n_chains, 4, beta, np.arange(1, n_chains + 1), gauge_sigma=0.1) as pc:
        rec = pc.run(3000, 0.005, cp, obs_every=10)
    x = rec[100:, :, 0] + 1j * rec[100:, :, 1]
    per_chain = x.mean(axis=0)
    err = per_chain.std() / np.sqrt(n_chains)
    assert abs(per_chain.mean() - exact) < 5 * abs(err) + 0.01, (per_chain.mean(), exact, err)
    assert np.isfinite(rec).all() and rec[:, :, 3].max() < 1e-12
