"""Pins of the oracle's adaptive Langevin step size: eps_n = eps min(1,
k_ref / K_max), K_max = max over links of |K|, |K|^2 = sum_a |K_a|^2,
K_a = -D_a S.  K_max is checked against central differences of the action
itself (the largest-drift link found independently), against the identity
sum_a |Tr(l_a X)|^2 = 2 |X - Tr X / 3|_F^2, and the step against the plain
step at the reduced eps."""
import numpy as np
import pytest
import scipy.linalg

import oracle as O
import lattice_inputs as LI

LAM = {a: O.gellmann(a) for a in range(1, 9)}


def _kmax_from_identity(X):
    tr = np.trace(X, axis1=-2, axis2=-1)[..., None, None] / 3.0
    Xp = X - tr * np.eye(3)
    return np.sqrt(2.0 * np.sum(np.abs(Xp) ** 2, axis=(-2, -1))).max()


def _k_fd(L, U, s, mu, beta, theta, delta=1e-5):
    """|K| of link (s, mu) from central differences of S along e^{i d l_a}."""
    k2 = 0.0
    for a in range(1, 9):
        vals = []
        for sign in (+1, -1):
            V = U.copy()
            V[s, mu] = scipy.linalg.expm(1j * sign * delta * LAM[a]) @ U[s, mu]
            vals.append(O.action(L, V, beta, theta))
        k2 += abs((vals[0] - vals[1]) / (2 * delta)) ** 2
    return np.sqrt(k2)


@pytest.mark.parametrize("L,beta,theta", [((2, 2, 2, 2), 5.5, 1.0), ((3, 2, 2, 3), 6.0, 0.5j)])
def test_kmax_is_the_largest_drift_of_the_action(L, beta, theta):
    U = LI.sl3c_lattice(L, seed=5, spread=0.2)
    _, e, kmax = O.cl_step_adaptive(L, U, beta, theta, 0.01, 0.0, 1, 0)
    X = O.drift(L, U, beta, theta)
    norms = np.sqrt(2.0 * np.sum(np.abs(X - np.trace(X, axis1=-2, axis2=-1)[..., None, None] / 3.0
                                        * np.eye(3)) ** 2, axis=(-2, -1)))
    s, mu = np.unravel_index(np.argmax(norms), norms.shape)
    k_fd = _k_fd(L, U, s, mu, beta, theta)
    assert abs(kmax - k_fd) < 1e-7 * max(1.0, kmax)
    assert abs(kmax - _kmax_from_identity(X)) < 1e-12 * kmax
    assert e == 0.01


def test_step_size_rule():
    L, beta, theta, eps, seed = (3, 3, 3, 3), 6.0, 1.0, 0.02, 4
    U = LI.sl3c_lattice(L, seed=9, spread=0.25)
    plain = O.cl_step(L, U, beta, theta, eps, seed, 3)
    # no reference, or a reference above K_max: the plain step, bit for bit
    for kref in (0.0, -1.0, 1e9):
        got, e, kmax = O.cl_step_adaptive(L, U, beta, theta, eps, kref, seed, 3)
        assert e == eps and np.array_equal(got, plain)
    # below K_max: eps_n K_max = eps k_ref, and the step is the plain step at eps_n
    kref = 0.25 * kmax
    got, e, k2 = O.cl_step_adaptive(L, U, beta, theta, eps, kref, seed, 3)
    assert k2 == kmax
    assert abs(e * kmax - eps * kref) < 1e-15
    assert np.array_equal(got, O.cl_step(L, U, beta, theta, e, seed, 3))
    # the update really is smaller: the drift part scales with eps_n, the noise with sqrt(eps_n)
    d_small = np.abs(got - U).max()
    d_full = np.abs(plain - U).max()
    assert d_small < d_full


def test_su3_links_keep_kmax_zero_at_zero_coupling():
    """beta = 0, theta = 0: S = 0, so K = 0 and eps_n = eps whatever k_ref."""
    L = (2, 2, 2, 2)
    U = LI.su3_lattice(L, seed=3)
    _, e, kmax = O.cl_step_adaptive(L, U, 0.0, 0.0, 0.01, 1e-6, 1, 0)
    assert kmax == 0.0 and e == 0.01
