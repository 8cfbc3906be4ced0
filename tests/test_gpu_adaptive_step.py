"""The adaptive Langevin step size on the GPU (drift pass with max |K|, step
size decided on the device, update from the stored drift) against the oracle,
and its special cases."""
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


def _lattice(L, beta, theta, prec, U, seed):
    lat = cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=seed, own_stream=True)
    lat.set_links(U)
    return lat


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_DF64])
@pytest.mark.parametrize("L,theta", [((4, 3, 4, 5), 1.0), ((3, 3, 3, 3), 0.5j), ((4, 4, 4, 4), 0.0)])
def test_adaptive_steps_against_the_oracle(L, theta, prec):
    beta, eps, seed = 6.0, 0.02, 21
    U = LI.sl3c_lattice(L, seed=4, spread=0.2)
    _, _, k0 = O.cl_step_adaptive(L, U, beta, theta, eps, 0.0, seed, 0)
    k_ref = 0.6 * k0  # the rule engages on the first steps
    with _lattice(L, beta, theta, prec, U, seed) as lat:
        lat.set_adaptive_step(k_ref)
        t_ref = 0.0
        for step in range(5):
            lat.step(eps, 1)
            U, e, k = O.cl_step_adaptive(L, U, beta, theta, eps, k_ref, seed, step)
            t_ref += e
            t, e_gpu, k_gpu = lat.langevin_time()
            assert abs(k_gpu - k) < 1e-12 * k, step
            assert abs(e_gpu - e) < 1e-14, step
            assert abs(t - t_ref) < 1e-13
            err = np.abs(lat.links() - U).max()
            assert err < 1e-12, (step, err)
        assert t_ref < 5 * eps  # some steps were shortened


def test_large_reference_is_the_plain_step_bit_for_bit():
    L, beta, theta, eps, seed = (4, 4, 3, 5), 6.0, 1.0, 0.01, 3
    U = LI.sl3c_lattice(L, seed=8, spread=0.2)
    for prec in (cl.CL_FP64, cl.CL_FP32_STORAGE, cl.CL_DF64):
        with _lattice(L, beta, theta, prec, U, seed) as a, _lattice(L, beta, theta, prec, U, seed) as b:
            b.set_adaptive_step(1e12)
            a.step(eps, 3)
            b.step(eps, 3)
            assert np.array_equal(a.links(), b.links())
            assert abs(a.langevin_time()[0] - 3 * eps) < 1e-15
            t, e, k = b.langevin_time()
            assert abs(t - 3 * eps) < 1e-15 and e == eps and k > 0


def test_fp32_adaptive_within_bound():
    L, beta, theta, eps, seed = (4, 4, 4, 4), 6.0, 1.0, 0.02, 5
    U = LI.sl3c_lattice(L, seed=6, spread=0.2)
    _, _, k0 = O.cl_step_adaptive(L, U, beta, theta, eps, 0.0, seed, 0)
    with _lattice(L, beta, theta, cl.CL_FP32_STORAGE, U, seed) as lat:
        lat.set_adaptive_step(0.5 * k0)
        lat.step(eps, 1)
        ref, e, k = O.cl_step_adaptive(L, U, beta, theta, eps, 0.5 * k0, seed, 0)
        _, e_gpu, k_gpu = lat.langevin_time()
        assert abs(k_gpu - k) < 1e-5 * k and abs(e_gpu - e) < 1e-5 * e
        assert np.abs(lat.links() - ref).max() < 2e-5


def test_adaptive_step_replays_in_a_graph():
    L, beta, theta, eps, seed = (4, 4, 4, 4), 6.0, 2.0, 0.02, 9
    U = LI.sl3c_lattice(L, seed=2, spread=0.2)
    cp = cl.make_cool(eps, 1.0, cl.CL_D2_MEANABS, n_min=1, n_max=4, tol_rel=0.05)
    with _lattice(L, beta, theta, cl.CL_FP64, U, seed) as a, _lattice(L, beta, theta, cl.CL_FP64, U, seed) as b:
        for lat in (a, b):
            lat.set_adaptive_step(5.0)
        b.capture_step(eps, cp)
        for _ in range(4):
            a.step(eps, 1)
            a.cool(cp)
        b.replay(4)
        assert np.array_equal(a.links(), b.links())
        assert a.langevin_time() == b.langevin_time()


def test_negative_reference_is_refused():
    with cl.Lattice((2, 2, 2, 2)) as lat:
        with pytest.raises(cl.CLError) as ei:
            lat.set_adaptive_step(-1.0)
        assert ei.value.status == cl.CL_ERR_INVALID
