"""FP64 CPU oracle for complex Langevin with adaptive gauge cooling (arXiv:1311.1056).

TEST INFRASTRUCTURE ONLY.  This is the independent checker of the CUDA path:
the test suite, the smoke check and the CPU-baseline leg of the benchmark are
the only code allowed to import it.  It shares nothing with the CUDA library.

Arrays: links are numpy complex128 of shape (V, 4, 3, 3) (site index
s = x0 + L0*(x1 + L1*(x2 + L2*x3)), direction mu = 0..3); per-site matrices
are (V, 3, 3); L is a 4-tuple of extents.  Each function cites the passage of
the paper it follows in the C++ source (oracle/oracle.cpp).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

D0, D1, D2_MEANABS, D2_RMS = 0, 1, 2, 3


class CoolParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("alpha", ctypes.c_double),
                ("mode", ctypes.c_int), ("n_min", ctypes.c_int), ("n_max", ctypes.c_int),
                ("tol_rel", ctypes.c_double), ("d_floor", ctypes.c_double),
                ("d_guard", ctypes.c_double), ("forced_sweeps", ctypes.c_int)]


class CoolReport(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("alpha_ad_last", ctypes.c_double),
                ("un_before", ctypes.c_double), ("un_after", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u64, u32, dbl, cint = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
        sig = {
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_normals": (None, [u64, u32, u32, u32, u32, cint, dp]),
            "or_normals_sites": (None, [u64, u32, u32, cint, u32, u32, cint, dp]),
            "or_gellmann": (None, [cint, dp]),
            "or_expm": (None, [dp, dp]),
            "or_inverse": (None, [dp, dp]),
            "or_det": (None, [dp, dp]),
            "or_cold_start": (cint, [ip, dp]),
            "or_hot_start": (cint, [ip, u64, dp]),
            "or_random_gauge": (cint, [ip, u64, dbl, dp]),
            "or_gauge_transform": (cint, [ip, dp, dp]),
            "or_observables": (cint, [ip, dp, dbl, dbl, dbl, dp]),
            "or_qdensity": (cint, [ip, dp, dp]),
            "or_action": (cint, [ip, dp, dbl, dbl, dbl, dp]),
            "or_drift": (cint, [ip, dp, dbl, dbl, dbl, dp]),
            "or_drift_at": (cint, [ip, dp, dbl, dbl, dbl, cint, i64p, dp]),
            "or_cl_step": (cint, [ip, dp, dbl, dbl, dbl, dbl, u64, u32]),
            "or_cl_step_adaptive": (cint, [ip, dp, dbl, dbl, dbl, dbl, dbl, u64, u32,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "or_cl_step_at": (cint, [ip, dp, dbl, dbl, dbl, dbl, u64, u32, cint, i64p, dp]),
            "or_step_sweep_at": (cint, [ip, dp, dbl, dbl, dbl, dbl, u64, u32, dbl, dbl, cint, i64p,
                                        dp, dp]),
            "or_cool_gradient": (cint, [ip, dp, dp]),
            "or_cool_sweep": (cint, [ip, dp, dbl, dbl]),
            "or_cool": (cint, [ip, dp, ctypes.POINTER(CoolParams), ctypes.POINTER(CoolReport)]),
            "or_trajectory": (cint, [ip, dp, dbl, dbl, dbl, dbl, u64, u32, cint,
                                     ctypes.POINTER(CoolParams), cint, dp]),
            "or_num_threads": (cint, []),
            "or_pauli": (None, [cint, dp]),
            "or_pc_cold": (cint, [cint, dp]),
            "or_pc_random_gauge": (cint, [cint, u64, dbl, dp]),
            "or_pc_action": (cint, [cint, dp, dbl, dbl, dp]),
            "or_pc_drift": (cint, [cint, dp, dbl, dbl, dp]),
            "or_pc_step": (cint, [cint, dp, dbl, dbl, dbl, u64, u32]),
            "or_pc_cool_gradient": (cint, [cint, dp, dp]),
            "or_pc_cool_sweep": (cint, [cint, dp, dbl, dbl]),
            "or_pc_cool": (cint, [cint, dp, ctypes.POINTER(CoolParams), ctypes.POINTER(CoolReport)]),
            "or_pc_observables": (cint, [cint, dp, dp]),
            "or_pc_trajectory": (cint, [cint, dp, dbl, dbl, dbl, u64, u32, cint,
                                        ctypes.POINTER(CoolParams), dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _L(L):
    arr = (ctypes.c_int * 4)(*[int(v) for v in L])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)), arr


def volume(L):
    return int(np.prod([int(v) for v in L]))


def _links(U, L):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    assert U.shape == (volume(L), 4, 3, 3), U.shape
    return U


def _check(rc, name):
    if rc != 0:
        raise ValueError("oracle %s failed with code %d" % (name, rc))


def num_threads():
    return lib().or_num_threads()


# ------------------------------------------------------------------ Philox
def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed, step, site, slot, stream, n_pairs):
    out = np.zeros(2 * n_pairs)
    lib().or_normals(seed, step, site, slot, stream, n_pairs, _dp(out))
    return out


def normals_sites(seed, step, site0, nsites, slot, stream, n_pairs):
    out = np.zeros((nsites, 2 * n_pairs))
    lib().or_normals_sites(seed, step, site0, nsites, slot, stream, n_pairs, _dp(out))
    return out


# ------------------------------------------------------------------ 3x3
def gellmann(a):
    out = np.zeros((3, 3), np.complex128)
    lib().or_gellmann(a, _dp(out))
    return out


def expm(A):
    A = np.ascontiguousarray(A, np.complex128)
    out = np.zeros((3, 3), np.complex128)
    lib().or_expm(_dp(A), _dp(out))
    return out


def inverse(A):
    A = np.ascontiguousarray(A, np.complex128)
    out = np.zeros((3, 3), np.complex128)
    lib().or_inverse(_dp(A), _dp(out))
    return out


def det(A):
    A = np.ascontiguousarray(A, np.complex128)
    out = np.zeros(2)
    lib().or_det(_dp(A), _dp(out))
    return complex(out[0], out[1])


# ------------------------------------------------------------------ lattice
def cold_start(L):
    U = np.zeros((volume(L), 4, 3, 3), np.complex128)
    Lp, _k = _L(L)
    _check(lib().or_cold_start(Lp, _dp(U)), "cold_start")
    return U


def hot_start(L, seed):
    U = np.zeros((volume(L), 4, 3, 3), np.complex128)
    Lp, _k = _L(L)
    _check(lib().or_hot_start(Lp, seed, _dp(U)), "hot_start")
    return U


def random_gauge(L, U, seed, sigma):
    U = _links(U, L).copy()
    Lp, _k = _L(L)
    _check(lib().or_random_gauge(Lp, seed, sigma, _dp(U)), "random_gauge")
    return U


def gauge_transform(L, U, Om):
    U = _links(U, L).copy()
    Om = np.ascontiguousarray(Om, np.complex128)
    assert Om.shape == (volume(L), 3, 3)
    Lp, _k = _L(L)
    _check(lib().or_gauge_transform(Lp, _dp(Om), _dp(U)), "gauge_transform")
    return U


OBS_NAMES = ("plaq_re", "plaq_im", "un", "q_re", "q_im", "sw_re", "sw_im", "s_re", "s_im",
             "max_det_dev")


def observables(L, U, beta=6.0, theta=0.0):
    U = _links(U, L)
    out = np.zeros(10)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_observables(Lp, _dp(U), beta, theta.real, theta.imag, _dp(out)), "observables")
    return dict(zip(OBS_NAMES, out.tolist()))


def qdensity(L, U):
    U = _links(U, L)
    out = np.zeros(2 * volume(L))
    Lp, _k = _L(L)
    _check(lib().or_qdensity(Lp, _dp(U), _dp(out)), "qdensity")
    return out[0::2] + 1j * out[1::2]


def action(L, U, beta, theta=0.0):
    U = _links(U, L)
    out = np.zeros(2)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_action(Lp, _dp(U), beta, theta.real, theta.imag, _dp(out)), "action")
    return complex(out[0], out[1])


def drift(L, U, beta, theta=0.0):
    U = _links(U, L)
    X = np.zeros_like(U)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_drift(Lp, _dp(U), beta, theta.real, theta.imag, _dp(X)), "drift")
    return X


def drift_at(L, U, beta, theta, links):
    U = _links(U, L)
    links = np.ascontiguousarray(links, np.int64)
    X = np.zeros((len(links), 3, 3), np.complex128)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_drift_at(Lp, _dp(U), beta, theta.real, theta.imag, len(links),
                             links.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(X)),
           "drift_at")
    return X


def cl_step(L, U, beta, theta, eps, seed, step):
    U = _links(U, L).copy()
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_cl_step(Lp, _dp(U), beta, theta.real, theta.imag, eps, seed, step), "cl_step")
    return U


def cl_step_adaptive(L, U, beta, theta, eps, k_ref, seed, step):
    """Returns (U', eps_n, K_max)."""
    U = _links(U, L).copy()
    theta = complex(theta)
    Lp, _k = _L(L)
    e, k = ctypes.c_double(), ctypes.c_double()
    _check(lib().or_cl_step_adaptive(Lp, _dp(U), beta, theta.real, theta.imag, eps, k_ref, seed, step,
                                     ctypes.byref(e), ctypes.byref(k)), "cl_step_adaptive")
    return U, e.value, k.value


def cl_step_at(L, U, beta, theta, eps, seed, step, links):
    U = _links(U, L)
    links = np.ascontiguousarray(links, np.int64)
    out = np.zeros((len(links), 3, 3), np.complex128)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_cl_step_at(Lp, _dp(U), beta, theta.real, theta.imag, eps, seed, step,
                               len(links), links.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               _dp(out)), "cl_step_at")
    return out


def step_sweep_at(L, U, beta, theta, eps, seed, step, eps_cool, alpha_ad, links):
    """U' after one CL step and U'' after one cooling sweep (alpha_ad fixed) at the given links."""
    U = _links(U, L)
    links = np.ascontiguousarray(links, np.int64)
    a = np.zeros((len(links), 3, 3), np.complex128)
    b = np.zeros((len(links), 3, 3), np.complex128)
    theta = complex(theta)
    Lp, _k = _L(L)
    _check(lib().or_step_sweep_at(Lp, _dp(U), beta, theta.real, theta.imag, eps, seed, step,
                                  eps_cool, alpha_ad, len(links),
                                  links.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(a),
                                  _dp(b)), "step_sweep_at")
    return a, b


def cool_gradient(L, U):
    U = _links(U, L)
    f = np.zeros((volume(L), 8))
    Lp, _k = _L(L)
    _check(lib().or_cool_gradient(Lp, _dp(U), _dp(f)), "cool_gradient")
    return f


def cool_sweep(L, U, eps, alpha_ad):
    U = _links(U, L).copy()
    Lp, _k = _L(L)
    _check(lib().or_cool_sweep(Lp, _dp(U), eps, alpha_ad), "cool_sweep")
    return U


def cool_params(eps, alpha=1.0, mode=D0, n_min=0, n_max=0, tol_rel=1e-3, d_floor=0.0,
                d_guard=1e-12, forced_sweeps=-1):
    return CoolParams(eps, alpha, mode, n_min, n_max, tol_rel, d_floor, d_guard, forced_sweeps)


def cool(L, U, params):
    U = _links(U, L).copy()
    rep = CoolReport()
    Lp, _k = _L(L)
    _check(lib().or_cool(Lp, _dp(U), ctypes.byref(params), ctypes.byref(rep)), "cool")
    return U, {"sweeps": rep.sweeps, "alpha_ad_last": rep.alpha_ad_last,
               "un_before": rep.un_before, "un_after": rep.un_after}


TRAJ_NAMES = OBS_NAMES + ("sweeps", "alpha_ad_last", "un_before", "un_after")


def trajectory(L, U, beta, theta, eps, seed, step0, n_steps, cool=None, obs_every=1):
    U = _links(U, L).copy()
    nrec = n_steps // obs_every if obs_every > 0 else 0
    out = np.zeros((max(nrec, 1), 14))
    theta = complex(theta)
    Lp, _k = _L(L)
    cp = ctypes.byref(cool) if cool is not None else None
    _check(lib().or_trajectory(Lp, _dp(U), beta, theta.real, theta.imag, eps, seed, step0,
                               n_steps, cp, obs_every, _dp(out)), "trajectory")
    return U, [dict(zip(TRAJ_NAMES, r.tolist())) for r in out[:nrec]]


# ------------------------------------------------- SU(2) Polyakov chain
# A chain is a complex128 array of shape (n, 2, 2); beta is complex.
def pauli(a):
    out = np.zeros((2, 2), np.complex128)
    lib().or_pauli(a, _dp(out))
    return out


def _chain(U):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    assert U.ndim == 3 and U.shape[1:] == (2, 2), U.shape
    return U


def pc_cold(n):
    U = np.zeros((n, 2, 2), np.complex128)
    _check(lib().or_pc_cold(n, _dp(U)), "pc_cold")
    return U


def pc_random_gauge(U, seed, sigma):
    U = _chain(U).copy()
    _check(lib().or_pc_random_gauge(len(U), seed, sigma, _dp(U)), "pc_random_gauge")
    return U


def pc_action(U, beta):
    U = _chain(U)
    b = complex(beta)
    out = np.zeros(2)
    _check(lib().or_pc_action(len(U), _dp(U), b.real, b.imag, _dp(out)), "pc_action")
    return complex(out[0], out[1])


def pc_drift(U, beta):
    U = _chain(U)
    b = complex(beta)
    out = np.zeros((len(U), 3), np.complex128)
    _check(lib().or_pc_drift(len(U), _dp(U), b.real, b.imag, _dp(out)), "pc_drift")
    return out


def pc_step(U, beta, eps, seed, step):
    U = _chain(U).copy()
    b = complex(beta)
    _check(lib().or_pc_step(len(U), _dp(U), b.real, b.imag, eps, seed, step), "pc_step")
    return U


def pc_cool_gradient(U):
    U = _chain(U)
    out = np.zeros((len(U), 3))
    _check(lib().or_pc_cool_gradient(len(U), _dp(U), _dp(out)), "pc_cool_gradient")
    return out


def pc_cool_sweep(U, eps, alpha_ad):
    U = _chain(U).copy()
    _check(lib().or_pc_cool_sweep(len(U), _dp(U), eps, alpha_ad), "pc_cool_sweep")
    return U


def pc_cool(U, params):
    U = _chain(U).copy()
    rep = CoolReport()
    _check(lib().or_pc_cool(len(U), _dp(U), ctypes.byref(params), ctypes.byref(rep)), "pc_cool")
    return U, {"sweeps": rep.sweeps, "alpha_ad_last": rep.alpha_ad_last,
               "un_before": rep.un_before, "un_after": rep.un_after}


PC_OBS_NAMES = ("tr_re", "tr_im", "un", "max_det_dev")


def pc_observables(U):
    U = _chain(U)
    out = np.zeros(4)
    _check(lib().or_pc_observables(len(U), _dp(U), _dp(out)), "pc_observables")
    return dict(zip(PC_OBS_NAMES, out.tolist()))


def pc_trajectory(U, beta, eps, seed, step0, n_steps, cool=None):
    """Returns (U, records): after every step tr_re, tr_im, un, max_det_dev, sweeps."""
    U = _chain(U).copy()
    b = complex(beta)
    rec = np.zeros((max(n_steps, 1), 5))
    cp = ctypes.byref(cool) if cool is not None else None
    _check(lib().or_pc_trajectory(len(U), _dp(U), b.real, b.imag, eps, seed, step0, n_steps, cp,
                                  _dp(rec)), "pc_trajectory")
    return U, rec[:n_steps]
