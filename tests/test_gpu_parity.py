"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Bars (FP64 form): 1e-12 max-abs on links after every step up to 10 steps
(with cooling), 1e-12 relative on drift matrices, gradients and
observables.  FP32-storage form: the bounds in FP32_TOL, derived from the
FP32 rounding of the link algebra (links are O(1); one update performs
~10^2 dependent roundings of 6e-8).

Inputs: seeded synthetic lattices from tests/lattice_inputs.py (random
SL(3,C) links, random gauge transformations) or the method's own seeded
starts; shapes include L = 2 (every loop wraps), a ragged 4x3x5x2 and
non-power-of-two extents.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import lattice_inputs as LI
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu

SHAPES = [(2, 2, 2, 2), (3, 3, 3, 3), (4, 3, 5, 2), (4, 4, 4, 4)]
FP32_TOL = {"links_1step": 2e-5, "drift_rel": 2e-5, "obs_rel": 2e-6, "grad_rel": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def lattice_from(U, L, beta=6.0, theta=0.0, prec=cl.CL_FP64, seed=1):
    lat = cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=seed)
    lat.set_links(U)
    return lat


def relerr(a, b):
    return np.abs(a - b).max() / max(1e-300, np.abs(b).max())


# ------------------------------------------------------------- starts
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (3, 4, 5, 2)])
def test_hot_start(L):
    with cl.Lattice(L, start=cl.CL_START_HOT, seed=7) as lat:
        assert np.abs(lat.links() - O.hot_start(L, 7)).max() < 1e-14


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (5, 3, 2, 4)])
def test_cold_start_random_gauge(L):
    with cl.Lattice(L, start=cl.CL_START_COLD, seed=1, gauge_sigma=0.05) as lat:
        ref = O.random_gauge(L, O.cold_start(L), 1, 0.05)
        assert np.abs(lat.links() - ref).max() < 1e-14


def test_links_roundtrip_and_step_counter():
    L = (3, 2, 4, 2)
    U = LI.sl3c_lattice(L, seed=2)
    with lattice_from(U, L) as lat:
        np.testing.assert_array_equal(lat.links(), U)
        assert lat.step_count == 0
        lat.step(0.01, 2)
        assert lat.step_count == 2


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE])
def test_links_roundtrip_through_pinned_host_memory(prec):
    """Page-locked host arrays are read and written in place by the layout
    kernels; pageable ones go through the staging buffer.  Both paths give
    the same links."""
    import torch
    L = (6, 4, 5, 3)
    V = 6 * 4 * 5 * 3
    U = LI.sl3c_lattice(L, seed=4, spread=0.3)
    with cl.Lattice(L, prec=prec) as lat:
        pin = torch.empty(V * 4 * 18, dtype=torch.float64, pin_memory=True)
        a_pin = pin.numpy().view(np.complex128).reshape(V, 4, 3, 3)
        a_pin[...] = U
        cl.cl_set_links(lat.h, a_pin)           # in place from pinned memory
        via_pin = lat.links()                   # out through the staging buffer
        lat.set_links(U)                        # in through the staging buffer
        via_stage = lat.links()
        np.testing.assert_array_equal(via_pin, via_stage)
        a_pin[...] = 0
        cl.cl_get_links(lat.h, V, a_pin)        # out in place to pinned memory
        np.testing.assert_array_equal(a_pin, via_stage)
        if prec == cl.CL_FP64:
            np.testing.assert_array_equal(via_stage, U)


# --------------------------------------------------------- drift and q_L
@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("beta,theta", [(5.8, 0.0), (0.0, 1.1 + 0.3j), (6.0, 2.0), (5.5, 0.7j)])
def test_drift_matches_oracle(L, beta, theta):
    U = LI.sl3c_lattice(L, seed=sum(L), spread=0.2)
    with lattice_from(U, L, beta=beta, theta=theta) as lat:
        X = lat.drift()
    ref = O.drift(L, U, beta, theta)
    assert relerr(X, ref) < 1e-12


@pytest.mark.parametrize("L", SHAPES)
def test_qdensity_and_observables(L):
    U = LI.sl3c_lattice(L, seed=3, spread=0.25)
    with lattice_from(U, L, beta=5.9, theta=0.8 + 0.1j) as lat:
        q = lat.qdensity()
        o = lat.observables()
    assert relerr(q, O.qdensity(L, U)) < 1e-12
    ref = O.observables(L, U, 5.9, 0.8 + 0.1j)
    for k, v in ref.items():
        tol = 1e-12 * max(1.0, abs(v)) if k != "max_det_dev" else 1e-14
        assert abs(o[k] - v) <= tol, (k, o[k], v)


def test_constant_flux_charge():
    """The closed-form pin of the oracle, checked on the GPU too."""
    L = (4, 6, 4, 6)
    n = {(0, 1): 2, (2, 3): -1, (0, 2): 1, (1, 3): 1, (0, 3): 1, (1, 2): -1}
    U = LI.constant_flux(L, n)
    phi = LI.flux_angles(L, n)
    s = {k: np.sin(v) for k, v in phi.items()}
    q_exact = (s[(0, 1)] * s[(2, 3)] - s[(0, 2)] * s[(1, 3)] + s[(0, 3)] * s[(1, 2)]) / (2 * np.pi**2)
    with lattice_from(U, L) as lat:
        assert np.abs(lat.qdensity() - q_exact).max() < 1e-13


# ------------------------------------------------------------ cooling
@pytest.mark.parametrize("L", SHAPES)
def test_cool_gradient(L):
    U = LI.sl3c_lattice(L, seed=5, spread=0.3)
    with lattice_from(U, L) as lat:
        f = lat.cool_gradient()
    assert relerr(f, O.cool_gradient(L, U)) < 1e-12


@pytest.mark.parametrize("mode", [cl.CL_D0, cl.CL_D1, cl.CL_D2_MEANABS, cl.CL_D2_RMS])
def test_cool_forced_sweeps(mode):
    L = (4, 3, 5, 2)
    U = LI.sl3c_lattice(L, seed=6, spread=0.2)
    cpar = dict(eps=0.01, alpha=0.9, mode=mode, forced_sweeps=3)
    with lattice_from(U, L) as lat:
        rep = lat.cool(cl.make_cool(**cpar))
        Ug = lat.links()
    Ur, rr = O.cool(L, U, O.cool_params(**cpar))
    assert np.abs(Ug - Ur).max() < 1e-12
    assert rep["sweeps"] == rr["sweeps"] == 3
    for k in ("alpha_ad_last", "un_before", "un_after"):
        assert abs(rep[k] - rr[k]) < 1e-12 * abs(rr[k]), k


def test_cool_adaptive_count():
    """The device-side stop rule takes the oracle's decisions (thresholds far
    from the measured values, so rounding cannot flip them)."""
    L = (4, 4, 4, 4)
    U = O.random_gauge(L, O.hot_start(L, 3), 1, 0.05)
    cpar = dict(eps=0.01, alpha=1.0, mode=cl.CL_D1, n_min=2, n_max=200, tol_rel=0.02, d_floor=1e-6)
    with lattice_from(U, L) as lat:
        rep = lat.cool(cl.make_cool(**cpar))
        Ug = lat.links()
    Ur, rr = O.cool(L, U, O.cool_params(**cpar))
    assert rep["sweeps"] == rr["sweeps"] and 2 <= rr["sweeps"] < 200
    assert np.abs(Ug - Ur).max() < 1e-12


def test_cooling_preserves_gauge_invariants():
    """Cooling is a gauge transformation (Sec. 2): plaquette, Q and S stay,
    the unitarity norm drops."""
    L = (4, 4, 4, 4)
    with cl.Lattice(L, beta=6.0, theta=1.0, start=cl.CL_START_HOT, seed=4, gauge_sigma=0.1) as lat:
        a = lat.observables()
        rep = lat.cool(cl.make_cool(0.01, 1.0, cl.CL_D0, forced_sweeps=50))
        b = lat.observables()
    for k in ("plaq_re", "plaq_im", "q_re", "q_im", "s_re", "s_im"):
        assert abs(a[k] - b[k]) < 1e-11 * max(1, abs(a[k])), k
    assert b["un"] < a["un"] and rep["un_after"] == pytest.approx(b["un"], rel=1e-14)


# ------------------------------------------------------------- CL step
@pytest.mark.parametrize("L", SHAPES)
@pytest.mark.parametrize("theta", [0.0, 1.0, 0.5 + 0.5j])
def test_one_cl_step(L, theta):
    U = LI.sl3c_lattice(L, seed=11, spread=0.15)
    with lattice_from(U, L, beta=6.0, theta=theta, seed=9) as lat:
        cl.cl_set_step(lat.h, 3)
        lat.step(0.01, 1)
        Ug = lat.links()
    Ur = O.cl_step(L, U, 6.0, theta, 0.01, 9, 3)
    assert np.abs(Ug - Ur).max() < 1e-13


@pytest.mark.parametrize("L,theta", [((4, 4, 4, 4), 1.0), ((4, 3, 5, 2), 2.0), ((2, 2, 2, 2), 0.5j)])
def test_ten_steps_with_cooling(L, theta):
    """Spec bar: links within 1e-12 of the oracle after each of 10
    steps, each followed by cooling (D_2, forced count)."""
    beta, eps, seed = 6.0, 0.005, 3
    U0 = O.random_gauge(L, O.hot_start(L, seed), seed, 0.05)
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D2_MEANABS, forced_sweeps=4)
    Ur = U0
    with lattice_from(U0, L, beta=beta, theta=theta, seed=seed) as lat:
        for step in range(10):
            lat.step(eps, 1)
            lat.cool(cl.make_cool(**cpar), want_report=False)
            Ur = O.cl_step(L, Ur, beta, theta, eps, seed, step)
            Ur, _ = O.cool(L, Ur, O.cool_params(**cpar))
            assert np.abs(lat.links() - Ur).max() < 1e-12, step


def test_golden_cfg0_trajectory():
    """4^4, beta 6, theta 0, cold start + random gauge, 20 steps at eps 0.01,
    5 sweeps alpha 1 (D_0): plaquette and unitarity norm of every step against
    the stored oracle values (tests/golden/cfg0_trajectory.json)."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg0_trajectory.json")))
    c = g["config"]
    with cl.Lattice(c["L"], beta=c["beta"], theta=c["theta"], seed=c["seed"],
                    gauge_sigma=c["sigma"]) as lat:
        cp = cl.make_cool(c["eps"], c["alpha"], cl.CL_D0, forced_sweeps=c["sweeps"])
        obs, reps = lat.trajectory(c["eps"], c["n_steps"], cp, obs_every=1)
    assert len(obs) == len(g["steps"]) == 20
    for o, r, ref in zip(obs, reps, g["steps"]):
        assert abs(o["plaq_re"] - ref["plaq_re"]) < 1e-12
        assert abs(o["un"] - ref["un"]) < 1e-12
        assert r["sweeps"] == 5


# ------------------------------------------------------ FP32-storage form
def test_fp32_storage_bounds():
    L = (4, 3, 5, 2)
    U = LI.sl3c_lattice(L, seed=21, spread=0.15)
    with lattice_from(U, L, beta=6.0, theta=1.0, prec=cl.CL_FP32_STORAGE, seed=2) as lat:
        assert relerr(lat.drift(), O.drift(L, U, 6.0, 1.0)) < FP32_TOL["drift_rel"]
        assert relerr(lat.cool_gradient(), O.cool_gradient(L, U)) < FP32_TOL["grad_rel"]
        o = lat.observables()
        ref = O.observables(L, U, 6.0, 1.0)
        for k in ("plaq_re", "un", "sw_re"):
            assert abs(o[k] - ref[k]) < FP32_TOL["obs_rel"] * max(1, abs(ref[k])), k
        lat.step(0.01, 1)
        Ug = lat.links()
        o = lat.observables()
    Ur = O.cl_step(L, U, 6.0, 1.0, 0.01, 2, 0)
    assert np.abs(Ug - Ur).max() < FP32_TOL["links_1step"]
    assert o["max_det_dev"] < 1e-6


# ------------------------------------------------------------- failures
def test_nonfinite_links_are_reported():
    L = (2, 2, 2, 2)
    U = LI.su3_lattice(L, 1)
    U[3, 2, 1, 1] = np.nan
    with lattice_from(U, L) as lat:
        with pytest.raises(cl.CLError) as e:
            lat.observables()
        assert e.value.status == cl.CL_ERR_NONFINITE
        with pytest.raises(cl.CLError) as e:
            lat.cool(cl.make_cool(0.01, 1.0, cl.CL_D0, forced_sweeps=2))
        assert e.value.status == cl.CL_ERR_NONFINITE


def test_invalid_cooling_arguments():
    with cl.Lattice((2, 2, 2, 2)) as lat:
        with pytest.raises(cl.CLError) as e:
            lat.cool(cl.make_cool(0.01, 1.0, 7, forced_sweeps=1))
        assert e.value.status == cl.CL_ERR_INVALID
        with pytest.raises(cl.CLError):
            lat.cool(cl.make_cool(0.01, 1.0, cl.CL_D0, n_min=5, n_max=2))
        with pytest.raises(cl.CLError):
            lat.step(-1.0, 1)
