"""Exact discrete one-link cooling model (Sec. 3), written from the algebra.

Test infrastructure only: it shares no code with the oracle or the CUDA path.

The model is a 1^4 lattice whose direction-0 link is an SL(2,C) block U
embedded in SL(3,C) and whose other links are the identity, so one cooling
sweep is U -> Omega U Omega^{-1} (Sec. 3).  For real c = Tr U / 2 the link is
gauge equivalent to SU(2), and up to a unitary change of frame it has the
canonical form

    U = diag(p, 1/p) R,   R = [[w, s], [-s, w]],   w, s real, w^2 + s^2 = 1,

with p >= 1 fixed by the distance d = Tr(U U^+ - 1)/2 = (p - 1/p)^2 / 2 and w
by the conserved trace, c = w (p + 1/p) / 2.  In that frame the algebra gives
in closed form

    H = U U^+ - U^+ U = h N,  h = (p^2 - p^-2) s,  N = [[s, -w], [-w, -s]],
    N^2 = 1,  sum_a f_a lambda_a = 4 H   (f_a = 2 Tr lambda_a H, eq. "eq:24"),
    Omega = exp(-eps alpha_ad 4 H) = cosh(t) - sinh(t) N,  t = 4 eps alpha_ad h,

so one sweep maps (d, c) to (d', c) with d' read off the real 2x2 product
Omega U Omega^{-1}.  Only invariants of the unitary frame enter: d, c, the
unitarity norm UN = 1 + d/6 of the 1^4 lattice (three identity links), D_1 =
UN and D_2(RMS) = sqrt(sum_a f_a^2 / 8) = sqrt(2) |h|.  (D_2 as the mean of
|f_a| depends on the frame and is left out.)  To first order in eps this is
eq. "eqgc" for N = 2 with Tr lambda_a lambda_b = 2 delta_ab:
d' - d = -32 eps alpha_ad (d + 2(1 - c^2)) d + O(eps^2).

`predict` applies the sweep-count reading of the adaptive rule (at least n_min
and at most n_max sweeps; stop once the norm fell by less than tol_rel of its
distance from 1, or that distance is below d_floor; no sweep while D <
d_guard) to this exact sequence.
"""
import math

import numpy as np

D0, D1, D2_RMS = 0, 1, 3


def canonical(d, c):
    """(p, w, s) of the canonical form for distance d >= 0 and real c."""
    r = math.sqrt(2.0 * d)
    p = 0.5 * (r + math.sqrt(2.0 * d + 4.0))
    w = 2.0 * c / (p + 1.0 / p)
    s = math.sqrt(max(0.0, 1.0 - w * w))
    return p, w, s


def block(d, c):
    """The canonical SL(2,C) block (real) for (d, c)."""
    p, w, s = canonical(d, c)
    return np.array([[p * w, p * s], [-s / p, w / p]])


def h_of(d, c):
    p, _w, s = canonical(d, c)
    return (p * p - 1.0 / (p * p)) * s


def sweep(d, c, eps_alpha):
    """Distance after one cooling sweep at eps * alpha_ad = eps_alpha."""
    p, w, s = canonical(d, c)
    U = block(d, c)
    N = np.array([[s, -w], [-w, -s]])
    t = 4.0 * eps_alpha * (p * p - 1.0 / (p * p)) * s
    Om = math.cosh(t) * np.eye(2) - math.sinh(t) * N
    Omi = math.cosh(t) * np.eye(2) + math.sinh(t) * N
    U1 = Om @ U @ Omi
    return 0.5 * (float(np.sum(U1 * U1)) - 2.0)


def un_of_d(d):
    """Unitarity norm (1/3)<Tr U U^+> of the 1^4 lattice with one block link."""
    return 1.0 + d / 6.0


def D_of(mode, d, c):
    if mode == D0:
        return 1.0
    if mode == D1:
        return un_of_d(d)
    if mode == D2_RMS:
        return math.sqrt(2.0) * abs(h_of(d, c))
    raise ValueError(mode)


def predict(d0, c, eps, alpha, mode, n_min, n_max, tol_rel, d_floor, d_guard=1e-12):
    """Sweep count, final UN and last alpha_ad of the adaptive rule on the
    exact sequence, with the smallest relative distance of any comparison the
    rule made from its threshold (a count is only pinned when that margin is
    far above rounding)."""
    d, k = d0, 0
    un_prev = None
    alpha_last = 0.0
    margin = math.inf
    uns = []

    def rel(a, b):
        return abs(a - b) / max(abs(a), abs(b), 1e-300)

    while True:
        un = un_of_d(d)
        uns.append(un)
        D = D_of(mode, d, c)
        stop = k >= n_max
        if k >= n_min:
            if d_floor > 0.0:
                margin = min(margin, rel(un - 1.0, d_floor))
            if un - 1.0 < d_floor:
                stop = True
            if k >= 1:
                lhs, rhs = un_prev - un, tol_rel * (un_prev - 1.0)
                if tol_rel > 0.0:
                    margin = min(margin, rel(lhs, rhs))
                if lhs < rhs:
                    stop = True
        if D < d_guard:
            stop = True
        if stop:
            return dict(sweeps=k, un_after=un, un_before=uns[0], alpha_ad_last=alpha_last,
                        margin=margin, uns=uns)
        alpha_ad = alpha / D
        d = sweep(d, c, eps * alpha_ad)
        alpha_last = alpha_ad
        un_prev = un
        k += 1


def lattice(d0, c, seed=3):
    """The 1^4 lattice (V, 4, 3, 3): the block for (d0, c) turned by a random
    SU(2) frame (the model depends on invariants only) as the direction-0
    link, identity elsewhere."""
    rng = np.random.default_rng(seed)
    z = rng.normal(size=4)
    z /= np.linalg.norm(z)
    W = np.array([[z[0] + 1j * z[1], z[2] + 1j * z[3]], [-z[2] + 1j * z[3], z[0] - 1j * z[1]]])
    U2 = W @ block(d0, c).astype(complex) @ W.conj().T
    U = np.zeros((1, 4, 3, 3), complex)
    U[0, :] = np.eye(3)
    U[0, 0, :2, :2] = U2
    return U


# Cases of the rule, each isolating one branch: (name, d0, c, eps, alpha,
# mode, n_min, n_max, tol_rel, d_floor).  The comment gives the count the
# exact sequence fixes by the branch the comment names.
CASES = [
    # linear regime: progress ~ 0.058 per sweep stays above tol, the floor stops
    ("floor", 0.5, 0.3, 1e-3, 1.0, D0, 0, 500, 1e-3, 1e-3),
    # nonlinear regime: progress falls from 0.15 through tol = 0.1
    ("progress", 3.0, 0.3, 1e-3, 1.0, D0, 0, 500, 0.1, 0.0),
    # n_min beyond the progress stop: exactly n_min
    ("n_min_above", 3.0, 0.3, 1e-3, 1.0, D0, 12, 500, 0.1, 0.0),
    # n_min before the progress stop: the progress count
    ("n_min_below", 3.0, 0.3, 1e-3, 1.0, D0, 5, 500, 0.1, 0.0),
    # n_min beyond the floor crossing: exactly n_min
    ("floor_n_min", 0.5, 0.3, 1e-3, 1.0, D0, 90, 500, 1e-3, 1e-3),
    # nothing triggers: n_max
    ("n_max", 3.0, 0.3, 1e-3, 1.0, D0, 0, 9, 0.0, 0.0),
    # D_1: alpha_ad = alpha / UN
    ("d1_progress", 3.0, 0.3, 1e-3, 1.0, D1, 0, 500, 0.075, 0.0),
    # D_2 (RMS): alpha_ad = alpha / (sqrt 2 |h|) makes the Omega angle
    # constant; the relative progress grows until a sweep overshoots the
    # minimum and the norm rises, which stops the rule
    ("d2rms_overshoot", 3.0, 0.3, 1e-3, 8.0, D2_RMS, 0, 500, 0.02, 0.0),
    ("d2rms_floor", 0.5, -0.6, 1e-3, 8.0, D2_RMS, 0, 500, 1e-4, 2e-2),
    # already unitary: D_2 = 0 is below the guard, no sweep
    ("guard", 0.0, 0.3, 1e-3, 1.0, D2_RMS, 3, 500, 1e-3, 0.0),
]
