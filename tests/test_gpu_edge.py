"""Edge cases: extents of 1 (every hop in that direction returns to the same
site, so a plaquette holds the same link twice), zero steps and zero sweeps,
and the largest lattices (16.8 M sites, where the drift-slot arrays pass
2^31 elements): a 4^4 random SL(3,C) field tiled periodically to 64^4 must
give the 4^4 oracle's drift, cooling gradient and intensive observables at
every one of its sites."""
import numpy as np
import pytest

import oracle as O
import lattice_inputs as LI
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def _from(U, L, beta=6.0, theta=0.0, prec=cl.CL_FP64, seed=1):
    lat = cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=seed)
    lat.set_links(U)
    return lat


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_DF64])
@pytest.mark.parametrize("L", [(1, 4, 4, 4), (2, 1, 3, 1), (1, 1, 1, 1), (3, 1, 1, 2)])
@pytest.mark.parametrize("theta", [0.0, 1.0])
def test_extents_of_one(L, theta, prec):
    U = LI.sl3c_lattice(L, seed=5, spread=0.2)
    beta, eps, seed = 6.0, 0.01, 4
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D1, forced_sweeps=2)
    with _from(U, L, beta, theta, prec=prec, seed=seed) as lat:
        X = lat.drift()
        f = lat.cool_gradient()
        o = lat.observables()
        lat.step(eps, 1)
        lat.cool(cl.make_cool(**cpar))
        U1 = lat.links()
    Xr = O.drift(L, U, beta, theta)
    assert np.abs(X - Xr).max() < 1e-12 * max(1.0, np.abs(Xr).max())
    fr = O.cool_gradient(L, U)
    assert np.abs(f - fr).max() < 1e-12 * max(1.0, np.abs(fr).max())
    ref = O.observables(L, U, beta, theta)
    for k in ("plaq_re", "plaq_im", "un", "q_re", "q_im", "s_re", "s_im"):
        assert abs(o[k] - ref[k]) < 1e-12 * max(1.0, abs(ref[k])), k
    Ur, _ = O.cool(L, O.cl_step(L, U, beta, theta, eps, seed, 0), O.cool_params(**cpar))
    assert np.abs(U1 - Ur).max() < 1e-12


def test_zero_steps_and_zero_sweeps():
    L = (4, 4, 4, 4)
    U = LI.sl3c_lattice(L, seed=2, spread=0.2)
    with _from(U, L, theta=1.0) as lat:
        lat.step(0.01, 0)
        assert lat.step_count == 0 and np.array_equal(lat.links(), lat.links())
        for cp in (cl.make_cool(0.01, 1.0, cl.CL_D1, n_min=0, n_max=0),
                   cl.make_cool(0.01, 1.0, cl.CL_D2_MEANABS, forced_sweeps=0)):
            rep = lat.cool(cp)
            assert rep["sweeps"] == 0
        assert np.abs(lat.links() - U).max() < 1e-15
        obs, reps = lat.trajectory(0.01, 0, None, obs_every=1)
        assert len(obs) == 0 and lat.step_count == 0


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP32_STORAGE, 3e-5), (cl.CL_FP64, 1e-12), (cl.CL_DF64, 1e-12)])
def test_largest_tiled_lattice(prec, tol):
    small, reps = (4, 4, 4, 4), (16, 16, 16, 16)
    L = tuple(a * r for a, r in zip(small, reps))  # 64^4 = 16,777,216 sites
    beta, theta = 6.0, 1.0
    Us = LI.sl3c_lattice(small, seed=8, spread=0.2)
    Xs = O.drift(small, Us, beta, theta)
    fs = O.cool_gradient(small, Us)
    ref = O.observables(small, Us, beta, theta)
    # site s = x0 + L0 (x1 + L1 (x2 + L2 x3)): tile along x0 fastest
    U = np.tile(Us.reshape(small[::-1] + (4, 3, 3)), reps[::-1] + (1, 1, 1)).reshape(-1, 4, 3, 3)
    with _from(U, L, beta, theta, prec=prec) as lat:
        del U
        X = lat.drift().reshape(L[::-1] + (4, 3, 3))
        scale = np.abs(Xs).max()
        for t in ((0, 0, 0, 0), (15, 7, 3, 9), (8, 15, 15, 0)):  # tiles across the index range
            sl = tuple(slice(4 * t[3 - i], 4 * t[3 - i] + 4) for i in range(4))
            err = np.abs(X[sl].reshape(-1, 4, 3, 3) - Xs).max()
            assert err < tol * scale, (t, err)
        del X
        f = lat.cool_gradient().reshape(L[::-1] + (8,))
        assert np.abs(f - np.tile(fs.reshape(small[::-1] + (8,)), reps[::-1] + (1,))).max() \
            < tol * max(1.0, np.abs(fs).max())
        del f
        o = lat.observables()
        nrep = int(np.prod(reps))
        for k in ("plaq_re", "plaq_im", "un"):
            assert abs(o[k] - ref[k]) < 10 * tol * max(1.0, abs(ref[k])), k
        for k in ("q_re", "q_im"):  # extensive: 4096 copies of the 4^4 charge
            assert abs(o[k] - nrep * ref[k]) < 10 * tol * nrep * max(1.0, abs(ref[k])), k
        lat.step(0.005, 1)
        lat.cool(cl.make_cool(0.005, 1.0, cl.CL_D1, forced_sweeps=1))
        o = lat.observables()
        assert np.isfinite([o[k] for k in o]).all() and o["un"] >= 1.0 - 1e-6
