"""The DF64 form (links as double-float pairs, link algebra on the FP32 pipe,
exponentials / noise / re-projection / reductions in FP64) against the FP64
oracle at the FP64 form's bars: drift, gradient and observables to 1e-12
relative, links within 1e-12 after each of 10 steps with cooling, and the
32^4 bench workload on sampled links."""
import numpy as np
import pytest

import oracle as O
import lattice_inputs as LI
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu

SHAPES = [(2, 2, 2, 2), (3, 3, 3, 3), (4, 3, 5, 2), (4, 4, 4, 4)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def _from(U, L, beta=6.0, theta=0.0, seed=1):
    lat = cl.Lattice(L, beta=beta, theta=theta, prec=cl.CL_DF64, seed=seed)
    lat.set_links(U)
    return lat


@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("theta", [0.0, 1.0, 0.5 + 0.5j])
def test_drift_gradient_observables(L, theta):
    U = LI.sl3c_lattice(L, seed=3, spread=0.2)
    with _from(U, L, 6.0, theta) as lat:
        X, f, o = lat.drift(), lat.cool_gradient(), lat.observables()
    Xr = O.drift(L, U, 6.0, theta)
    assert np.abs(X - Xr).max() < 1e-12 * np.abs(Xr).max()
    fr = O.cool_gradient(L, U)
    assert np.abs(f - fr).max() < 1e-12 * max(1.0, np.abs(fr).max())
    ref = O.observables(L, U, 6.0, theta)
    for k in ("plaq_re", "plaq_im", "un", "q_re", "q_im", "s_re", "s_im"):
        assert abs(o[k] - ref[k]) < 1e-12 * max(1.0, abs(ref[k])), k


@pytest.mark.parametrize("L,theta", [((4, 4, 4, 4), 1.0), ((4, 3, 5, 2), 2.0), ((2, 2, 2, 2), 0.5j)])
def test_ten_steps_with_cooling(L, theta):
    beta, eps, seed = 6.0, 0.005, 3
    U0 = O.random_gauge(L, O.hot_start(L, seed), seed, 0.05)
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D2_MEANABS, forced_sweeps=4)
    Ur = U0
    with _from(U0, L, beta, theta, seed) as lat:
        for step in range(10):
            lat.step(eps, 1)
            lat.cool(cl.make_cool(**cpar), want_report=False)
            Ur = O.cl_step(L, Ur, beta, theta, eps, seed, step)
            Ur, _ = O.cool(L, Ur, O.cool_params(**cpar))
            assert np.abs(lat.links() - Ur).max() < 1e-12, step


def test_32x4_step_and_sweep_sampled():
    L = (32, 32, 32, 32)
    beta, theta, eps, seed = 6.2, 1.0, 0.005, 1
    U0 = O.hot_start(L, seed)
    with cl.Lattice(L, beta=beta, theta=theta, prec=cl.CL_DF64, seed=seed, start=cl.CL_START_HOT) as lat:
        start_err = np.abs(lat.links() - U0).max()
        lat.step(eps, 1)
        U1 = lat.links()
        lat.cool(cl.make_cool(eps, 1.0, cl.CL_D0, forced_sweeps=1))
        U2 = lat.links()
    assert start_err < 1e-11  # the FP64 Haar start stored as hi + lo (R18 conditioning)
    links = LI.sample_links(LI.volume(L), 48, seed=32)
    a, b = O.step_sweep_at(L, U0, beta, theta, eps, seed, 0, eps, 1.0, links)
    tol = max(1e-12, 10 * start_err)
    assert np.abs(U1.reshape(-1, 3, 3)[links] - a).max() < tol
    assert np.abs(U2.reshape(-1, 3, 3)[links] - b).max() < tol


def test_df64_tracks_fp64_on_the_bench_workload():
    """16^4, beta 6.2, theta 1, Haar start, 10 steps of [CL step + 10 D_1
    sweeps]: the DF64 links stay within 1e-11 of the FP64 ones."""
    L = (16, 16, 16, 16)
    cp = cl.make_cool(0.005, 1.0, cl.CL_D1, forced_sweeps=10)
    out = []
    for prec in (cl.CL_FP64, cl.CL_DF64):
        with cl.Lattice(L, beta=6.2, theta=1.0, prec=prec, seed=1, start=cl.CL_START_HOT) as lat:
            for _ in range(10):
                lat.step(0.005, 1)
                lat.cool(cp, want_report=False)
            out.append((lat.links(), lat.observables()))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-11
    for k in ("plaq_re", "un", "q_re", "q_im"):
        assert abs(out[0][1][k] - out[1][1][k]) < 1e-11 * max(1.0, abs(out[0][1][k])), k


def test_df64_in_graphs_batches_and_checkpoints():
    L = (4, 4, 4, 6)
    cp = cl.make_cool(0.01, 1.0, cl.CL_D2_MEANABS, n_min=1, n_max=6, tol_rel=0.05)
    mk = lambda: cl.Lattice(L, beta=6.0, theta=1.0, prec=cl.CL_DF64, seed=5, start=cl.CL_START_HOT,
                            gauge_sigma=0.05, own_stream=True)
    with mk() as a, mk() as b, mk() as c:
        for _ in range(3):
            a.step(0.01, 1)
            a.cool(cp)
        b.capture_step(0.01, cp)
        b.replay(3)
        with cl.Batch([c], 0.01, [cp]) as bt:
            bt.run(3)
        assert np.array_equal(a.links(), b.links()) and np.array_equal(a.links(), c.links())
        ck = a.save_state()
        with mk() as d:
            d.load_state(ck)
            for lat in (a, d):
                lat.step(0.01, 2)
                lat.cool(cp)
            assert np.array_equal(a.links(), d.links())
