"""Pins of the SU(2) Polyakov-chain oracle (Sec. 3, Sec. 4, eq. "eq:s"):
the Pauli algebra, the drift against central differences of the action, the
cooling step against eq. "eqgc" (d' - d = -eps alpha f_a^2 / N to first
order), the exact one-link fixed points of Sec. 3 (d -> 0 when c is real,
d -> |c|^2 - 1 + sqrt(1 - c^2 - c*^2 + |c|^4) otherwise), gauge invariance of
the action and of (1/2) Tr(U_1 ... U_N), and the exact expectation value
<(1/2) Tr(U_1 ... U_N)> = I_2(beta) / I_1(beta) of the one-link model the
chain reduces to."""
import numpy as np
import pytest
import scipy.linalg
import scipy.special

import oracle as O

SIG = {a: O.pauli(a) for a in (1, 2, 3)}


def random_sl2c(r, n, spread=0.3):
    out = np.zeros((n, 2, 2), np.complex128)
    for k in range(n):
        w = r.normal(size=3) + 1j * spread * r.normal(size=3)
        out[k] = scipy.linalg.expm(1j * sum(w[a - 1] * SIG[a] for a in (1, 2, 3)))
    return out


def test_pauli_algebra():
    for a in (1, 2, 3):
        for b in (1, 2, 3):
            assert abs(np.trace(SIG[a] @ SIG[b]) - 2.0 * (a == b)) < 1e-15
    assert np.allclose(SIG[1] @ SIG[2] - SIG[2] @ SIG[1], 2j * SIG[3])
    assert np.allclose(SIG[2] @ SIG[3] - SIG[3] @ SIG[2], 2j * SIG[1])


@pytest.mark.parametrize("n,beta", [(1, 1.3), (3, 0.8 + 0.6j), (6, 2.0 - 1.0j)])
def test_drift_is_minus_the_derivative_of_the_action(n, beta):
    r = np.random.default_rng(n)
    U = random_sl2c(r, n)
    K = O.pc_drift(U, beta)
    d = 1e-5
    for k in range(n):
        for a in (1, 2, 3):
            vals = []
            for sg in (+1, -1):
                V = U.copy()
                V[k] = scipy.linalg.expm(1j * sg * d * SIG[a]) @ U[k]
                vals.append(O.pc_action(V, beta))
            DS = (vals[0] - vals[1]) / (2 * d)
            assert abs(K[k, a - 1] + DS) < 1e-8 * max(1.0, abs(DS)), (k, a)


def test_cooling_step_follows_eqgc():
    """One sweep at small eps changes d = UN - 1 by -eps alpha sum f^2 / N_c
    (N_c = 2) summed over the sites, per link of the chain (eq. "eqgc")."""
    r = np.random.default_rng(7)
    for n in (1, 4):
        U = random_sl2c(r, n, spread=0.4)
        f = O.pc_cool_gradient(U)
        eps, alpha = 1e-7, 1.0
        d0 = O.pc_observables(U)["un"] - 1.0
        d1 = O.pc_observables(O.pc_cool_sweep(U, eps, alpha))["un"] - 1.0
        pred = -alpha * np.sum(f ** 2) / 2.0 / n
        assert abs((d1 - d0) / eps - pred) < 1e-4 * abs(pred), n


def _one_link(c_re, c_im, r):
    """An SL(2,C) matrix with (1/2) Tr U = c, not normal (a random similarity)."""
    c = complex(c_re, c_im)
    lam = c + np.sqrt(c * c - 1.0)
    D = np.diag([lam, 1.0 / lam])
    G = scipy.linalg.expm(sum((r.normal() + 0.5j * r.normal()) * SIG[a] for a in (1, 2, 3)) * 0.4)
    return (G @ D @ np.linalg.inv(G))[None]


def test_one_link_fixed_points_of_sec3():
    r = np.random.default_rng(3)
    cp = O.cool_params(0.002, 1.0, O.D0, forced_sweeps=40000)
    # c = c*: gauge equivalent to SU(2), d -> 0
    U = _one_link(0.6, 0.0, r)
    V, _ = O.pc_cool(U, cp)
    assert O.pc_observables(V)["un"] - 1.0 < 1e-10
    # c != c*: d -> |c|^2 - 1 + sqrt(1 - c^2 - c*^2 + |c|^4)
    for c in (0.6 + 0.3j, 1.4 - 0.5j):
        U = _one_link(c.real, c.imag, r)
        V, _ = O.pc_cool(U, cp)
        cc = np.trace(V[0]) / 2
        assert abs(cc - c) < 1e-12  # cooling is a similarity: c is kept
        a2 = abs(c) ** 2
        d_inf = a2 - 1.0 + np.sqrt(1.0 - c * c - np.conj(c) ** 2 + a2 * a2).real
        assert abs(O.pc_observables(V)["un"] - 1.0 - d_inf) < 1e-9, c


def test_gauge_invariance_and_cooling_back_to_su2():
    n = 8
    U = O.pc_random_gauge(O.pc_cold(n), 5, 0.2)
    o = O.pc_observables(U)
    assert abs(o["tr_re"] - 1.0) < 1e-12 and abs(o["tr_im"]) < 1e-12 and o["un"] > 1.01
    r = np.random.default_rng(2)
    W = random_sl2c(r, n)
    b = 1.1 + 0.4j
    G = O.pc_random_gauge(W, 9, 0.3)
    assert abs(O.pc_action(G, b) - O.pc_action(W, b)) < 1e-12 * abs(O.pc_action(W, b))
    V, rep = O.pc_cool(U, O.cool_params(0.01, 1.0, O.D1, forced_sweeps=3000))
    assert O.pc_observables(V)["un"] - 1.0 < 1e-9
    assert abs(O.pc_observables(V)["tr_re"] - 1.0) < 1e-10


def test_real_beta_from_su2_stays_in_su2():
    n = 5
    U = O.pc_cold(n)
    U, rec = O.pc_trajectory(U, 1.7, 0.01, 3, 0, 50)
    assert np.abs(rec[:, 2] - 1.0).max() < 1e-13
    assert np.abs(rec[:, 1]).max() < 1e-13
    assert np.abs(O.pc_cool_gradient(U)).max() < 1e-12
    for k in range(n):
        assert np.allclose(U[k] @ U[k].conj().T, np.eye(2), atol=1e-13)


@pytest.mark.parametrize("beta", [1.5, 1.0 + 0.5j])
def test_exact_answer_of_the_one_link_model(beta):
    """<(1/2) Tr(U_1..U_4)> = I_2(beta) / I_1(beta), with adaptive cooling
    (D_2), within five standard errors of the mean over 20 blocks."""
    exact = scipy.special.iv(2, beta) / scipy.special.iv(1, beta)
    U = O.pc_random_gauge(O.pc_cold(4), 1, 0.1)
    cp = O.cool_params(0.01, 1.0, O.D2_MEANABS, n_min=1, n_max=10, tol_rel=0.01)
    U, rec = O.pc_trajectory(U, beta, 0.005, 1, 0, 40000, cp)
    x = rec[2000:, 0] + 1j * rec[2000:, 1]
    blocks = x[: len(x) // 20 * 20].reshape(20, -1).mean(axis=1)
    err = blocks.std() / np.sqrt(20)
    assert abs(x.mean() - exact) < 5 * err + 0.01, (x.mean(), exact, err)
