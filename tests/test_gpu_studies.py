"""The studies of Sec. 3-5 on the GPU kernels: gauge cooling of a single
link converges exponentially (Sec. 3), longer chains converge more slowly
(Sec. 4, Fig. "Nlink"), the D_2 rule reaches a given distance in fewer sweeps
than the fixed strength at first (Sec. 4), and in the theta scan the action
is real for theta_L^2 <= 0 (links stay in SU(3), Q_L real) but not for real
theta_L (Sec. 5)."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O
from paper_1311_1056_gb300 import build, cl, studies

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def test_one_link_cools_exponentially():
    sig = {a: O.pauli(a) for a in (1, 2, 3)}
    G = scipy.linalg.expm(0.3 * (0.8 * sig[1] + 0.5j * sig[2] - 0.4 * sig[3]))
    c = 0.6
    lam = c + 1j * np.sqrt(1 - c * c)
    U = G @ np.diag([lam, 1 / lam]) @ np.linalg.inv(G)  # (1/2) Tr U = 0.6: equivalent to SU(2)
    cp = cl.make_cool(0.01, 1.0, cl.CL_D0, forced_sweeps=1)
    with cl.PolyakovChains(1, 1, 1.0, [1]) as pc:
        pc.set_links(U[None, None])
        d = pc.run(400, 0.0, cp, obs_every=1)[:, 0, 2] - 1.0
    assert d[0] > 1e-2 and d[-1] < 1e-10
    # exponential: log d falls linearly (at a constant rate) once d is small,
    # down to the rounding level
    idx = np.nonzero((d > 1e-11) & (d < 1e-4))[0]
    assert len(idx) >= 10 and np.all(np.diff(idx) == 1)
    rate = -np.diff(np.log(d[idx]))
    assert rate.std() < 0.05 * rate.mean()


def test_longer_chains_cool_more_slowly():
    reach = {}
    for n in (10, 100, 1000):
        d = studies.chain_cooling(n, "D0", alpha=1.0, eps=0.01, sweeps=1500)[:, 0]
        reach[n] = studies.summarize(d)["first_sweep_below"]["1e-05"]
        if n == 1000:
            late = studies.summarize(d)["loglog_slope_last_decade"]
    assert reach[10] < reach[100] <= reach[1000] + 50
    assert -2.5 < late < -1.0  # a power law, not the single link's exponential


def test_long_chain_decay_is_a_power_law_near_three_halves():
    """Sec. 4: on a long chain the distance decays asymptotically like
    t^(-3/2) under the fixed-strength cooling (N = 1000, sweeps 500-5000)."""
    d = studies.chain_cooling(1000, "D0", alpha=1.0, eps=0.01, sweeps=5000)[:, 0]
    x = np.log(np.arange(500, 5000) + 1.0)
    slope = np.polyfit(x, np.log(d[500:5000]), 1)[0]
    assert -1.75 < slope < -1.25, slope


def test_d2_reaches_the_first_decades_sooner():
    d0 = studies.summarize(studies.chain_cooling(1000, "D0", sweeps=300)[:, 0])
    d2 = studies.summarize(studies.chain_cooling(1000, "D2", alpha=1.0, sweeps=300)[:, 0])
    assert d2["first_sweep_below"]["0.001"] < d0["first_sweep_below"]["0.001"]


def test_theta_scan_real_and_imaginary_theta():
    # D_1 cooling with at least one sweep per step keeps real-action chains at SU(3) to
    # rounding (the unitary directions are unstable under CL and rounding seeds them)
    cp = cl.make_cool(0.005, 1.0, cl.CL_D1, n_min=1, n_max=10, tol_rel=0.01)
    res = studies.theta_scan(betas=(6.0,), theta2=(0.0, 1.0, -1.0), n_steps=400, every=20, cool=cp)
    by = {r["theta2"]: r for r in res}
    for t2 in (0.0, -1.0):  # real action: the links stay in SU(3), where q_L is real
        assert np.abs(by[t2]["un"] - 1.0).max() < 1e-12
        assert np.abs(by[t2]["q"].imag).max() < 1e-10
    # complex action: the links leave SU(3) and Q_L acquires an imaginary part
    assert (by[1.0]["un"] - 1.0).max() > 1e-8
    assert np.abs(by[1.0]["q"].imag).max() > 1e-4
    for r in res:
        assert np.isfinite(r["plaq"]).all() and r["langevin_time"] > 0


def test_theta_dependence_of_q_at_small_theta():
    """<q_L> = i theta_L chi_L + O(theta^3) (Sec. 5): on 6^4 at beta = 6.1 over
    Langevin time ~60, Im Q grows with real theta, Re Q falls with theta =
    i phi, and both slopes are the same chi within the errors."""
    res = studies.theta_scan(betas=(6.1,), theta2=(1.0, 4.0, -1.0, -4.0), n_steps=16000, every=20)
    q = {}
    for r in res:
        x = r["q"][len(r["q"]) // 4:]
        nb = 8
        b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
        q[r["theta2"]] = (x.mean(), np.abs(b - b.mean()).std() / np.sqrt(nb))
        assert np.isfinite(x).all()
    (q1, e1), (q2, e2) = q[1.0], q[4.0]
    (p1, f1), (p2, f2) = q[-1.0], q[-4.0]
    assert q1.imag > 3 * e1 and q2.imag > q1.imag
    assert p1.real < -3 * f1 and p2.real < p1.real
    assert abs(q1.imag + p1.real) < 4 * np.hypot(e1, f1)  # the same chi for real and imaginary theta


# ------------------------------------------------- SU(3) lattices (NEXT-2)
def _oracle_lattice_cooling(L, mode, alpha, eps, sweeps, sigma, seed):
    """d after each of `sweeps` single-sweep cooling calls of the oracle, from
    the cold start transformed by the oracle's random SL(3,C) gauge
    transformation (the same Philox stream the library's start uses)."""
    U = O.random_gauge(L, O.cold_start(L), seed, sigma)
    d = []
    for _ in range(sweeps):
        U, rep = O.cool(L, U, O.cool_params(eps, alpha, mode, forced_sweeps=1))
        d.append(rep["un_after"] - 1.0)
    return np.array(d)


@pytest.mark.parametrize("mode,omode", [("D0", O.D0), ("D1", O.D1), ("D2", O.D2_MEANABS)])
def test_lattice_cooling_series_matches_oracle(mode, omode):
    """Sec. 4 on an SU(3) lattice: the distance d = UN - 1 after each of the
    first 20 sweeps of the study (one cooling call per sweep) equals the
    oracle's, to 1e-12, for D_0, D_1 and D_2 (4 x 3 x 5 x 2, every loop wraps)."""
    L, alpha, eps, sigma, seed = (4, 3, 5, 2), 1.0, 0.01, 0.1, 3
    d_gpu = studies.lattice_cooling(L, mode, alpha=alpha, eps=eps, sweeps=20, sigma=sigma, seed=seed)
    d_or = _oracle_lattice_cooling(L, omode, alpha, eps, 20, sigma, seed)
    assert d_or[0] > 1e-3
    assert np.abs(d_gpu - d_or).max() < 1e-12, np.abs(d_gpu - d_or).max()


def test_lattice_cooling_d0_d1_d2():
    """Sec. 4 on an 8^4 SU(3) lattice (cold start moved off SU(3) by a random
    SL(3,C) transformation): with the fixed strength (D_0) and the norm
    normalisation (D_1) the distance falls every sweep and keeps falling past
    1e-5; D_1 ~ D_0 here because UN ~ 1.  The normalised-gradient rule D_2
    takes a step of fixed size whatever |f| is, so at alpha = 1 it stalls on a
    plateau above 1e-4 (it never reaches 1e-5); at alpha = 0.1 it descends
    more slowly and stalls on a plateau two orders of magnitude lower (the
    step shrinks with alpha)."""
    L, eps, sweeps = (8, 8, 8, 8), 0.01, 120
    d0 = studies.lattice_cooling(L, "D0", alpha=1.0, eps=eps, sweeps=sweeps)
    d1 = studies.lattice_cooling(L, "D1", alpha=1.0, eps=eps, sweeps=sweeps)
    d2 = studies.lattice_cooling(L, "D2", alpha=1.0, eps=eps, sweeps=sweeps)
    d2s = studies.lattice_cooling(L, "D2", alpha=0.1, eps=eps, sweeps=300)
    s0, s1, s2 = (studies.summarize(d) for d in (d0, d1, d2))
    # D_0 / D_1: monotone decrease, both thresholds reached, nearly in step
    for d in (d0, d1):
        live = d[d > 1e-13]
        assert np.all(np.diff(live) < 0)
    assert s0["first_sweep_below"]["1e-05"] is not None and s1["first_sweep_below"]["1e-05"] is not None
    assert abs(s0["first_sweep_below"]["0.001"] - s1["first_sweep_below"]["0.001"]) <= 1
    # D_2 at alpha = 1: never below 1e-5, and flat over the last half (a plateau)
    assert s2["first_sweep_below"]["1e-05"] is None
    tail = d2[sweeps // 2:]
    assert tail.min() > 1e-4 and tail.max() < 3 * tail.min()
    # a smaller alpha: slower descent, then a much lower plateau
    s2s = studies.summarize(d2s)
    assert s2s["first_sweep_below"]["0.001"] > 3 * s2["first_sweep_below"]["0.001"]
    assert d2s[150:].max() < 0.1 * tail.min()
