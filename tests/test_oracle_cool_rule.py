"""Pin of the oracle's cooling sweep and adaptive sweep-count rule against
the exact discrete one-link model (Sec. 3 reduced to the invariants d and c;
`one_link_model.py` derives it).

The paper fixes alpha_ad = alpha / D (Sec. 4) but no stop rule; the reading
taken is: at least n_min and at most n_max sweeps, stop once the unitarity
norm fell by less than tol_rel of its distance from 1 or that distance is
below d_floor, no sweep while D < d_guard.  Here the norm's whole sequence is
known in closed form, so each branch of that rule has an exact count: a
reversed progress test, an off-by-one at n_min or n_max, a floor compared the
wrong way or a D taken from the wrong sweep moves a count and fails.
"""
import math

import pytest

import oracle as O
import one_link_model as M

L1 = (1, 1, 1, 1)


@pytest.mark.parametrize("d0,c", [(0.5, 0.3), (3.0, -0.6), (0.02, 0.9)])
def test_one_link_sweep_is_exact(d0, c):
    """Sec. 3 one-link model: the oracle's unitarity norm after k forced
    sweeps equals the closed-form sequence, for k up to 60."""
    eps, alpha = 2e-3, 0.7
    U = M.lattice(d0, c, seed=11)
    d = d0
    for k in range(61):
        if k in (1, 2, 7, 60):
            _, rep = O.cool(L1, U, O.cool_params(eps, alpha, O.D0, forced_sweeps=k))
            assert rep["sweeps"] == k
            assert abs(rep["un_after"] - M.un_of_d(d)) < 1e-13, (k, rep["un_after"], M.un_of_d(d))
        d = M.sweep(d, c, eps * alpha)


def test_closed_form_matches_eqgc_to_first_order():
    """The closed form reduces to eq. "eqgc" for N = 2: with Tr l_a l_b =
    2 delta_ab, (d' - d)/eps -> -32 alpha (d + 2(1 - c^2)) d (four times the
    printed N = 2 right-hand side, the reading of that equation taken
    throughout), and the linearised rate is 64 alpha (1 - c^2)."""
    for d, c in ((0.3, 0.2), (2.0, -0.5), (1e-4, 0.7)):
        alpha = 0.9
        r = [(M.sweep(d, c, e * alpha) - d) / e for e in (2e-6, 1e-6)]
        rate = 2 * r[1] - r[0]
        exact = -32 * alpha * (d + 2 * (1 - c * c)) * d
        assert abs(rate - exact) < 1e-6 * abs(exact)


def test_d2_rms_closed_form():
    """D_2 (RMS) of the model, sqrt(2)|h|, against the oracle's gradient."""
    for d0, c in ((0.5, 0.3), (3.0, -0.6)):
        f = O.cool_gradient(L1, M.lattice(d0, c, seed=5))[0]
        assert abs(math.sqrt((f**2).mean()) - M.D_of(M.D2_RMS, d0, c)) < 1e-12 * M.D_of(M.D2_RMS, d0, c)


@pytest.mark.parametrize("case", M.CASES, ids=[c[0] for c in M.CASES])
def test_adaptive_rule_count(case):
    """Each branch of the sweep-count rule stops the oracle at the sweep the
    exact sequence fixes; UN before / after and the last alpha_ad agree."""
    _name, d0, c, eps, alpha, mode, n_min, n_max, tol, d_floor = case
    P = M.predict(d0, c, eps, alpha, mode, n_min, n_max, tol, d_floor)
    assert P["margin"] > 1e-4  # far from any threshold: rounding cannot flip it
    _, rep = O.cool(L1, M.lattice(d0, c), O.cool_params(eps, alpha, mode, n_min, n_max, tol, d_floor))
    assert rep["sweeps"] == P["sweeps"]
    assert abs(rep["un_before"] - P["un_before"]) < 1e-14
    assert abs(rep["un_after"] - P["un_after"]) < 1e-13
    assert abs(rep["alpha_ad_last"] - P["alpha_ad_last"]) <= 1e-10 * max(1.0, P["alpha_ad_last"])


def test_rule_counts_are_distinct():
    """The cases separate the branches: their counts differ where a mistake
    in one branch would otherwise be hidden by another."""
    n = {c[0]: M.predict(*c[1:])["sweeps"] for c in M.CASES}
    assert n["progress"] > 1 and n["floor"] > 1  # a reversed progress test stops at 1
    assert n["n_min_above"] == 12 and n["floor_n_min"] == 90 and n["n_max"] == 9
    assert n["n_min_below"] == n["progress"] and n["guard"] == 0
    assert n["d1_progress"] not in (n["progress"], 1)
