"""ctypes binding of libcl.so (include/cl.h), same names as the C functions.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Importing works without a GPU; calling into the
library needs libcl.so (built by paper_1311_1056_gb300/build.py) and raises
if it is missing -- there is no CPU fallback.

Host link arrays are numpy complex128 of shape (V, 4, 3, 3) (the AoS layout
of cl.h); `cl_get_links_device` / `cl_set_links_device` take device pointers
(e.g. torch.Tensor.data_ptr() of a float64 CUDA tensor of 2*V*4*9 elements).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcl.so")

CL_OK, CL_ERR_INVALID, CL_ERR_OOM, CL_ERR_CUDA, CL_ERR_NONFINITE, CL_ERR_RUNAWAY, CL_ERR_TIMEOUT = range(7)
CL_FP64, CL_FP32_STORAGE, CL_DF64 = 0, 1, 2
CL_START_COLD, CL_START_HOT = 0, 1
CL_D0, CL_D1, CL_D2_MEANABS, CL_D2_RMS = 0, 1, 2, 3
CL_TUNE_CLOVER, CL_TUNE_FORCE, CL_TUNE_UPDATE, CL_TUNE_OMEGA, CL_TUNE_APPLY = range(5)
CL_NTUNE = 5
TUNE_CANDIDATES = (32, 64, 128, 256)


class cl_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("beta", ctypes.c_double),
                ("theta_re", ctypes.c_double), ("theta_im", ctypes.c_double),
                ("prec", ctypes.c_int), ("seed", ctypes.c_uint64), ("start", ctypes.c_int),
                ("gauge_sigma", ctypes.c_double)]


class cl_cool_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("alpha", ctypes.c_double), ("mode", ctypes.c_int),
                ("n_min", ctypes.c_int), ("n_max", ctypes.c_int), ("tol_rel", ctypes.c_double),
                ("d_floor", ctypes.c_double), ("d_guard", ctypes.c_double),
                ("forced_sweeps", ctypes.c_int)]


class cl_obs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("plaq_re", "plaq_im", "un", "q_re", "q_im", "sw_re",
                                               "sw_im", "s_re", "s_im", "max_det_dev")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class cl_cool_report(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("alpha_ad_last", ctypes.c_double),
                ("un_before", ctypes.c_double), ("un_after", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class cl_request(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 4), ("beta", ctypes.c_double), ("theta_re", ctypes.c_double),
                ("theta_im", ctypes.c_double), ("eps", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("start", ctypes.c_int), ("gauge_sigma", ctypes.c_double),
                ("tag", ctypes.c_int64)]


class cl_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("max_slots", ctypes.c_int),
                ("prec", ctypes.c_int), ("chunk_steps", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("cool_enabled", ctypes.c_int), ("cool", cl_cool_params),
                ("blocks_from_autotune", ctypes.c_int), ("k_ref", ctypes.c_double),
                ("runaway_un", ctypes.c_double)]


class cl_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int64), ("status", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("obs", cl_obs), ("last_cool", cl_cool_report), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {"tag": self.tag, "status": self.status, "n_steps": self.n_steps,
                "obs": self.obs.as_dict(), "last_cool": self.last_cool.as_dict(),
                "t_submit": self.t_submit, "t_admit": self.t_admit, "t_done": self.t_done}


class cl_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("runaways", ctypes.c_int64),
                ("active", ctypes.c_int), ("queued", ctypes.c_int), ("pooled", ctypes.c_int),
                ("peak_active", ctypes.c_int), ("bytes_in_use", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class CLError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, _status_str(status), _last_error()))


_lib = None
_P = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "cl_init_lattice": (ctypes.c_int, [ctypes.POINTER(cl_params), _P, ctypes.POINTER(_P)]),
    "cl_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int]),
    "cl_cool": (ctypes.c_int, [_P, ctypes.POINTER(cl_cool_params), ctypes.POINTER(cl_cool_report)]),
    "cl_observables": (ctypes.c_int, [_P, ctypes.POINTER(cl_obs)]),
    "cl_trajectory": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(cl_cool_params), ctypes.c_int,
                                     ctypes.POINTER(cl_obs), ctypes.POINTER(cl_cool_report),
                                     ctypes.c_double]),
    "cl_get_links": (ctypes.c_int, [_P, _dp]),
    "cl_set_links": (ctypes.c_int, [_P, _dp]),
    "cl_get_links_device": (ctypes.c_int, [_P, _P]),
    "cl_set_links_device": (ctypes.c_int, [_P, _P]),
    "cl_get_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "cl_set_step": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "cl_drift": (ctypes.c_int, [_P, _dp]),
    "cl_cool_gradient": (ctypes.c_int, [_P, _dp]),
    "cl_qdensity": (ctypes.c_int, [_P, _dp]),
    "cl_noise_sample": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _dp]),
    "cl_selftest_convert": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "cl_selftest_box_muller": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_int64)]),
    "cl_wait": (ctypes.c_int, [_P, ctypes.c_double]),
    "cl_batch_wait": (ctypes.c_int, [_P, ctypes.c_double]),
    "cl_batch_set_fused": (ctypes.c_int, [_P, ctypes.c_int]),
    "cl_batch_get_fused": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "cl_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "cl_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "cl_get_timing": (ctypes.c_int, [_P, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "cl_synchronize": (ctypes.c_int, [_P]),
    "cl_free": (None, [_P]),
    "cl_observables_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, _P, _P]),
    "cl_cool_last_report": (ctypes.c_int, [_P, ctypes.POINTER(cl_cool_report)]),
    "cl_set_adaptive_step": (ctypes.c_int, [_P, ctypes.c_double]),
    "cl_get_langevin_time": (ctypes.c_int, [_P, _dp, _dp, _dp]),
    "cl_set_blocks": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "cl_get_blocks": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "cl_autotune": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(cl_cool_params), ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]),
    "cl_pchain_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.c_double, _P, ctypes.POINTER(_P)]),
    "cl_pchain_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(cl_cool_params),
                                      ctypes.c_int, _dp]),
    "cl_pchain_get_links": (ctypes.c_int, [_P, _dp]),
    "cl_pchain_set_links": (ctypes.c_int, [_P, _dp]),
    "cl_pchain_get_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "cl_pchain_free": (None, [_P]),
    "cl_state_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "cl_save_state": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_size_t]),
    "cl_load_state": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_size_t]),
    "cl_stream_create": (ctypes.c_int, [ctypes.POINTER(_P)]),
    "cl_stream_destroy": (ctypes.c_int, [_P]),
    "cl_capture_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(cl_cool_params)]),
    "cl_replay": (ctypes.c_int, [_P, ctypes.c_int]),
    "cl_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), _dp,
                                       ctypes.POINTER(cl_cool_params), ctypes.c_int,
                                       ctypes.POINTER(_P)]),
    "cl_batch_run": (ctypes.c_int, [_P, ctypes.c_int]),
    "cl_batch_add": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.POINTER(cl_cool_params)]),
    "cl_batch_remove": (ctypes.c_int, [_P, _P]),
    "cl_batch_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "cl_batch_synchronize": (ctypes.c_int, [_P]),
    "cl_batch_free": (None, [_P]),
    "cl_reset_lattice": (ctypes.c_int, [_P, ctypes.POINTER(cl_params)]),
    "cl_lattice_bytes": (ctypes.c_int, [ctypes.POINTER(cl_params), ctypes.POINTER(ctypes.c_size_t)]),
    "cl_server_create": (ctypes.c_int, [ctypes.POINTER(cl_server_config), ctypes.POINTER(_P)]),
    "cl_server_clock": (ctypes.c_double, [_P]),
    "cl_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(cl_request), ctypes.c_double]),
    "cl_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(cl_result), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "cl_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(cl_server_stats)]),
    "cl_server_run_trace": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(cl_request), _dp,
                                           ctypes.POINTER(cl_result)]),
    "cl_server_free": (None, [_P]),
    "cl_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "cl_last_error": (ctypes.c_char_p, []),
    "cl_version": (ctypes.c_int, []),
}


def load(path=LIB_PATH):
    """Load libcl.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libcl.so not found at %s: run paper_1311_1056_gb300/build.py "
                               "(or __graft_entry__.build()) first" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _status_str(s):
    return load().cl_status_str(s).decode()


def _last_error():
    return load().cl_last_error().decode()


def _check(s, where):
    if s != CL_OK:
        raise CLError(s, where)


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    assert a.size * 2 == n, (a.shape, n)
    return a


# ----------------------------------------------------------------- C names
def cl_init_lattice(params, stream=0):
    h = _P()
    _check(load().cl_init_lattice(ctypes.byref(params), _P(stream or None), ctypes.byref(h)),
           "cl_init_lattice")
    return h


def cl_step(lat, eps, n_steps):
    _check(load().cl_step(lat, eps, n_steps), "cl_step")


def cl_cool(lat, cp, want_report=True):
    rep = cl_cool_report()
    _check(load().cl_cool(lat, ctypes.byref(cp), ctypes.byref(rep) if want_report else None), "cl_cool")
    return rep.as_dict() if want_report else None


def cl_cool_last_report(lat):
    rep = cl_cool_report()
    _check(load().cl_cool_last_report(lat, ctypes.byref(rep)), "cl_cool_last_report")
    return rep.as_dict()


def cl_set_adaptive_step(lat, k_ref):
    _check(load().cl_set_adaptive_step(lat, k_ref), "cl_set_adaptive_step")


def cl_get_langevin_time(lat):
    """Returns (t, eps_last, kmax_last)."""
    t, e, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().cl_get_langevin_time(lat, ctypes.byref(t), ctypes.byref(e), ctypes.byref(k)),
           "cl_get_langevin_time")
    return t.value, e.value, k.value


def cl_set_blocks(lat, blocks):
    b = (ctypes.c_int * CL_NTUNE)(*[int(v) for v in blocks])
    _check(load().cl_set_blocks(lat, b), "cl_set_blocks")


def cl_get_blocks(lat):
    b = (ctypes.c_int * CL_NTUNE)()
    _check(load().cl_get_blocks(lat, b), "cl_get_blocks")
    return list(b)


def cl_autotune(lat, eps, cp, reps=3, use_cache=True, want_table=False):
    """Returns (blocks, table): table[c][f] = mean ms per step of family f at
    block size TUNE_CANDIDATES[c] (None unless want_table)."""
    b = (ctypes.c_int * CL_NTUNE)()
    ms = np.zeros((len(TUNE_CANDIDATES), CL_NTUNE)) if want_table else None
    _check(load().cl_autotune(lat, eps, ctypes.byref(cp), reps, int(use_cache), b,
                              ms.ctypes.data_as(_dp) if want_table else None), "cl_autotune")
    return list(b), ms


def cl_reset_lattice(lat, params):
    _check(load().cl_reset_lattice(lat, ctypes.byref(params)), "cl_reset_lattice")


def cl_lattice_bytes(params):
    b = ctypes.c_size_t()
    _check(load().cl_lattice_bytes(ctypes.byref(params), ctypes.byref(b)), "cl_lattice_bytes")
    return b.value


def make_request(L, beta, theta, eps, n_steps, seed, start=CL_START_COLD, gauge_sigma=0.0, tag=0):
    L = tuple(int(v) for v in (L if hasattr(L, "__len__") else (L,) * 4))
    th = complex(theta)
    return cl_request((ctypes.c_int * 4)(*L), beta, th.real, th.imag, eps, int(n_steps), seed, start,
                      gauge_sigma, tag)


def make_server_config(hbm_budget_bytes=150e9, max_slots=64, prec=CL_FP32_STORAGE, chunk_steps=8,
                       use_graphs=True, cool=None, blocks_from_autotune=True, k_ref=0.0, runaway_un=0.0):
    return cl_server_config(hbm_budget_bytes, max_slots, prec, chunk_steps, int(use_graphs),
                            int(cool is not None), cool if cool is not None else cl_cool_params(),
                            int(blocks_from_autotune), k_ref, runaway_un)


def cl_server_create(cfg):
    h = _P()
    _check(load().cl_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cl_server_create")
    return h


def cl_server_clock(srv):
    return load().cl_server_clock(srv)


def cl_server_submit(srv, req, t_submit=-1.0):
    _check(load().cl_server_submit(srv, ctypes.byref(req), t_submit), "cl_server_submit")


def cl_server_poll(srv, max_out=64):
    out = (cl_result * max_out)()
    n = ctypes.c_int()
    _check(load().cl_server_poll(srv, out, max_out, ctypes.byref(n)), "cl_server_poll")
    return [out[i].as_dict() for i in range(n.value)]


def cl_server_stats_get(srv):
    st = cl_server_stats()
    _check(load().cl_server_stats_get(srv, ctypes.byref(st)), "cl_server_stats_get")
    return st.as_dict()


def cl_server_run_trace(srv, reqs, arrivals):
    n = len(reqs)
    arr = (cl_request * max(n, 1))(*reqs)
    t = np.ascontiguousarray(arrivals, dtype=np.float64)
    out = (cl_result * max(n, 1))()
    _check(load().cl_server_run_trace(srv, n, arr, t.ctypes.data_as(_dp), out), "cl_server_run_trace")
    return [out[i].as_dict() for i in range(n)]


def cl_server_free(srv):
    load().cl_server_free(srv)


def cl_state_size(lat):
    n = ctypes.c_size_t()
    _check(load().cl_state_size(lat, ctypes.byref(n)), "cl_state_size")
    return n.value


def cl_save_state(lat):
    """The chain's checkpoint as bytes."""
    buf = np.zeros(cl_state_size(lat), np.uint8)
    _check(load().cl_save_state(lat, buf.ctypes.data, buf.size), "cl_save_state")
    return buf.tobytes()


def cl_load_state(lat, data):
    buf = np.frombuffer(data, np.uint8).copy()
    _check(load().cl_load_state(lat, buf.ctypes.data, buf.size), "cl_load_state")


def cl_stream_create():
    h = _P()
    _check(load().cl_stream_create(ctypes.byref(h)), "cl_stream_create")
    return h.value


def cl_stream_destroy(stream):
    _check(load().cl_stream_destroy(_P(stream)), "cl_stream_destroy")


def cl_capture_step(lat, eps, cp=None):
    _check(load().cl_capture_step(lat, eps, ctypes.byref(cp) if cp is not None else None),
           "cl_capture_step")


def cl_replay(lat, n_steps):
    _check(load().cl_replay(lat, n_steps), "cl_replay")


def cl_batch_create(lats, eps, cps=None):
    n = len(lats)
    hs = (_P * n)(*[ctypes.cast(h, _P) for h in lats])
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,)))
    cp_arr = (cl_cool_params * n)(*cps) if cps is not None else None
    b = _P()
    _check(load().cl_batch_create(n, hs, e.ctypes.data_as(_dp), cp_arr, int(cps is not None),
                                  ctypes.byref(b)), "cl_batch_create")
    return b


def cl_batch_run(batch, n_steps):
    _check(load().cl_batch_run(batch, n_steps), "cl_batch_run")


def cl_batch_add(batch, lat, eps, cp=None):
    _check(load().cl_batch_add(batch, lat, eps, ctypes.byref(cp) if cp is not None else None), "cl_batch_add")


def cl_batch_remove(batch, lat):
    _check(load().cl_batch_remove(batch, lat), "cl_batch_remove")


def cl_batch_size(batch):
    n = ctypes.c_int()
    _check(load().cl_batch_size(batch, ctypes.byref(n)), "cl_batch_size")
    return n.value


def cl_batch_synchronize(batch):
    _check(load().cl_batch_synchronize(batch), "cl_batch_synchronize")


def cl_wait(lat, timeout_s):
    """True when the lattice's work has finished, False on CL_ERR_TIMEOUT."""
    st = load().cl_wait(lat, timeout_s)
    if st == CL_ERR_TIMEOUT:
        return False
    _check(st, "cl_wait")
    return True


def cl_batch_wait(batch, timeout_s):
    st = load().cl_batch_wait(batch, timeout_s)
    if st == CL_ERR_TIMEOUT:
        return False
    _check(st, "cl_batch_wait")
    return True


def cl_batch_set_fused(batch, fused):
    _check(load().cl_batch_set_fused(batch, 1 if fused else 0), "cl_batch_set_fused")


def cl_batch_get_fused(batch):
    v = ctypes.c_int()
    _check(load().cl_batch_get_fused(batch, ctypes.byref(v)), "cl_batch_get_fused")
    return bool(v.value)


def cl_batch_free(batch):
    load().cl_batch_free(batch)


def cl_observables(lat, check=True):
    o = cl_obs()
    s = load().cl_observables(lat, ctypes.byref(o))
    if check:
        _check(s, "cl_observables")
    return o.as_dict()


def cl_trajectory(lat, eps, n_steps, cp=None, obs_every=0, runaway_un=0.0):
    nrec = n_steps // obs_every if obs_every > 0 else 0
    obs = (cl_obs * max(nrec, 1))()
    rep = (cl_cool_report * max(nrec, 1))()
    _check(load().cl_trajectory(lat, eps, n_steps, ctypes.byref(cp) if cp is not None else None,
                                obs_every, obs, rep, runaway_un), "cl_trajectory")
    return [obs[k].as_dict() for k in range(nrec)], [rep[k].as_dict() for k in range(nrec)]


def cl_get_links(lat, V, out=None):
    if out is None:
        out = np.empty((V, 4, 3, 3), np.complex128)
    _check(load().cl_get_links(lat, out.ctypes.data_as(_dp)), "cl_get_links")
    return out


def cl_set_links(lat, U):
    U = _f64(U, 2 * U.size)
    _check(load().cl_set_links(lat, U.ctypes.data_as(_dp)), "cl_set_links")


def cl_get_links_device(lat, dev_ptr):
    _check(load().cl_get_links_device(lat, _P(dev_ptr)), "cl_get_links_device")


def cl_set_links_device(lat, dev_ptr):
    _check(load().cl_set_links_device(lat, _P(dev_ptr)), "cl_set_links_device")


def cl_get_step(lat):
    v = ctypes.c_uint64()
    _check(load().cl_get_step(lat, ctypes.byref(v)), "cl_get_step")
    return v.value


def cl_set_step(lat, step):
    _check(load().cl_set_step(lat, step), "cl_set_step")


def cl_drift(lat, V):
    out = np.empty((V, 4, 3, 3), np.complex128)
    _check(load().cl_drift(lat, out.ctypes.data_as(_dp)), "cl_drift")
    return out


def cl_cool_gradient(lat, V):
    out = np.empty((8, V))
    _check(load().cl_cool_gradient(lat, out.ctypes.data_as(_dp)), "cl_cool_gradient")
    return out.T.copy()  # (V, 8), like the oracle


def noise_sample(prec, seed, step, mu, site0, nsites):
    """The 8 standard normals of links (site0 .. site0 + nsites - 1, mu) at
    `step`, as the kernels of form `prec` draw them: array (nsites, 8)."""
    out = np.empty((max(nsites, 0), 8))
    _check(load().cl_noise_sample(prec, seed, step, mu, site0, nsites, out.ctypes.data_as(_dp)),
           "cl_noise_sample")
    return out


def cl_selftest_convert(seed, n):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().cl_selftest_convert(seed, n, ctypes.byref(a), ctypes.byref(b)), "cl_selftest_convert")
    return a.value, b.value


def cl_selftest_box_muller(seed, n):
    """(ulp_ln, ulp_sincos): largest distances of the FP64 noise's ln and
    sincospi from CUDA's log and sincospi over n generated uniforms."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().cl_selftest_box_muller(seed, n, ctypes.byref(a), ctypes.byref(b)), "cl_selftest_box_muller")
    return a.value, b.value


def cl_qdensity(lat, V):
    out = np.empty(2 * V)
    _check(load().cl_qdensity(lat, out.ctypes.data_as(_dp)), "cl_qdensity")
    return out[0::2] + 1j * out[1::2]


def cl_launch_count(lat):
    v = ctypes.c_int64()
    _check(load().cl_launch_count(lat, ctypes.byref(v)), "cl_launch_count")
    return v.value


PHASES = ("clover", "update", "cool_grad", "cool_rule", "cool_omega", "cool_apply", "obs", "force",
          "cool_grad_omega")


def cl_set_timing(lat, on):
    _check(load().cl_set_timing(lat, 1 if on else 0), "cl_set_timing")


def cl_get_timing(lat):
    ms = (ctypes.c_double * len(PHASES))()
    n = (ctypes.c_int64 * len(PHASES))()
    _check(load().cl_get_timing(lat, ms, n), "cl_get_timing")
    return {p: (ms[i], n[i]) for i, p in enumerate(PHASES)}


def cl_synchronize(lat):
    _check(load().cl_synchronize(lat), "cl_synchronize")


def cl_free(lat):
    if lat:
        load().cl_free(lat)


def cl_observables_noalloc(dev_links, L, beta, theta, dev_out, stream=0):
    """Observables of caller-owned device links (float64 AoS, 2*V*4*9 values)
    into caller-owned device memory (10 float64), with no device allocation
    in the library; enqueued on `stream`, nothing synchronised."""
    theta = complex(theta)
    Larr = (ctypes.c_int * 4)(*[int(v) for v in L])
    _check(load().cl_observables_noalloc(_P(dev_links), Larr, beta, theta.real, theta.imag,
                                         _P(dev_out), _P(stream or None)), "cl_observables_noalloc")


def cl_status_str(s):
    return _status_str(s)


def cl_last_error():
    return _last_error()


def cl_version():
    return load().cl_version()


# ----------------------------------------------------------- convenience
def make_params(L, beta=6.0, theta=0.0, prec=CL_FP64, seed=1, start=CL_START_COLD, gauge_sigma=0.0):
    theta = complex(theta)
    p = cl_params()
    for mu in range(4):
        p.L[mu] = int(L[mu])
    p.beta = beta
    p.theta_re, p.theta_im = theta.real, theta.imag
    p.prec, p.seed, p.start, p.gauge_sigma = prec, seed, start, gauge_sigma
    return p


def make_cool(eps, alpha=1.0, mode=CL_D0, n_min=0, n_max=0, tol_rel=1e-3, d_floor=0.0,
              d_guard=1e-12, forced_sweeps=-1):
    return cl_cool_params(eps, alpha, mode, n_min, n_max, tol_rel, d_floor, d_guard, forced_sweeps)


class PolyakovChains:
    """Owning wrapper of cl_pchain: n_chains SU(2) Polyakov chains of n_links
    links (beta: one complex value or one per chain; seeds: one per chain).
    Links as complex128 arrays of shape (n_chains, n_links, 2, 2)."""

    def __init__(self, n_chains, n_links, beta, seeds, gauge_sigma=0.0, stream=0):
        self.n_chains, self.n_links = int(n_chains), int(n_links)
        b = np.broadcast_to(np.asarray(beta, dtype=np.complex128), (self.n_chains,))
        bb = np.ascontiguousarray(np.stack([b.real, b.imag], axis=1))
        sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
        assert sd.shape == (self.n_chains,)
        self.h = None
        h = _P()
        _check(load().cl_pchain_create(self.n_chains, self.n_links, bb.ctypes.data_as(_dp),
                                       sd.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), gauge_sigma,
                                       _P(stream or None), ctypes.byref(h)), "cl_pchain_create")
        self.h = h

    def run(self, n_steps, eps, cp=None, obs_every=0):
        """Returns records of shape (n_steps // obs_every, n_chains, 5):
        tr_re, tr_im, un, max_det_dev, sweeps (empty when obs_every = 0)."""
        nrec = n_steps // obs_every if obs_every > 0 else 0
        out = np.zeros((max(nrec, 1), self.n_chains, 5))
        _check(load().cl_pchain_run(self.h, n_steps, eps, ctypes.byref(cp) if cp is not None else None,
                                    obs_every, out.ctypes.data_as(_dp)), "cl_pchain_run")
        return out[:nrec]

    def links(self):
        out = np.zeros((self.n_chains, self.n_links, 2, 2), np.complex128)
        _check(load().cl_pchain_get_links(self.h, out.ctypes.data_as(_dp)), "cl_pchain_get_links")
        return out

    def set_links(self, U):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        assert U.shape == (self.n_chains, self.n_links, 2, 2)
        _check(load().cl_pchain_set_links(self.h, U.ctypes.data_as(_dp)), "cl_pchain_set_links")

    @property
    def step_count(self):
        v = ctypes.c_uint64()
        _check(load().cl_pchain_get_step(self.h, ctypes.byref(v)), "cl_pchain_get_step")
        return v.value

    def close(self):
        if getattr(self, "h", None):
            load().cl_pchain_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owning wrapper of cl_server (see make_server_config)."""

    def __init__(self, cfg):
        self.h = None
        self.h = cl_server_create(cfg)

    def clock(self):
        return cl_server_clock(self.h)

    def submit(self, req, t_submit=-1.0):
        cl_server_submit(self.h, req, t_submit)

    def poll(self, max_out=64):
        return cl_server_poll(self.h, max_out)

    def stats(self):
        return cl_server_stats_get(self.h)

    def run_trace(self, reqs, arrivals):
        return cl_server_run_trace(self.h, reqs, arrivals)

    def drain(self, n, sleep=1e-4):
        """Poll until n results have come back; returns them."""
        import time
        out = []
        while len(out) < n:
            got = self.poll()
            out.extend(got)
            if not got:
                time.sleep(sleep)
        return out

    def close(self):
        if getattr(self, "h", None):
            cl_server_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper of cl_batch: one graph launch advances every chain by
    one step.  The Lattice objects must outlive it and have distinct,
    non-default streams (Lattice(..., own_stream=True))."""

    def __init__(self, lats, eps, cps=None, fused=None):
        """fused: None keeps the library's default (fused where the members
        allow it), True / False sets the mode."""
        self.lats = list(lats)
        self.h = None
        self.h = cl_batch_create([l.h for l in self.lats], eps, cps)
        if fused is not None:
            cl_batch_set_fused(self.h, fused)

    def run(self, n_steps=1):
        cl_batch_run(self.h, n_steps)

    def add(self, lat, eps, cp=None):
        cl_batch_add(self.h, lat.h, eps, cp)
        self.lats.append(lat)

    def remove(self, lat):
        cl_batch_remove(self.h, lat.h)
        self.lats.remove(lat)

    def __len__(self):
        return cl_batch_size(self.h)

    def synchronize(self):
        cl_batch_synchronize(self.h)

    def set_fused(self, fused):
        cl_batch_set_fused(self.h, fused)

    @property
    def fused(self):
        return cl_batch_get_fused(self.h)

    def close(self):
        if getattr(self, "h", None):
            cl_batch_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    """Owning wrapper: frees the device lattice when closed or collected."""

    def __init__(self, L, beta=6.0, theta=0.0, prec=CL_FP64, seed=1, start=CL_START_COLD,
                 gauge_sigma=0.0, stream=0, own_stream=False):
        self.L = tuple(int(v) for v in L)
        self.V = int(np.prod(self.L))
        self.params = make_params(L, beta, theta, prec, seed, start, gauge_sigma)
        self.h = None
        self._own = cl_stream_create() if own_stream else None
        self.stream = self._own if own_stream else stream
        self.h = cl_init_lattice(self.params, self.stream)

    def step(self, eps, n=1):
        cl_step(self.h, eps, n)

    def cool(self, cp, want_report=True):
        return cl_cool(self.h, cp, want_report)

    def observables(self):
        return cl_observables(self.h)

    def last_cool_report(self):
        return cl_cool_last_report(self.h)

    def set_adaptive_step(self, k_ref):
        cl_set_adaptive_step(self.h, k_ref)

    def langevin_time(self):
        return cl_get_langevin_time(self.h)

    def save_state(self):
        return cl_save_state(self.h)

    def load_state(self, data):
        cl_load_state(self.h, data)

    def autotune(self, eps, cp, reps=3, use_cache=True, want_table=False):
        return cl_autotune(self.h, eps, cp, reps, use_cache, want_table)

    def blocks(self):
        return cl_get_blocks(self.h)

    def set_blocks(self, blocks):
        cl_set_blocks(self.h, blocks)

    def capture_step(self, eps, cp=None):
        cl_capture_step(self.h, eps, cp)

    def replay(self, n_steps=1):
        cl_replay(self.h, n_steps)

    def synchronize(self):
        cl_synchronize(self.h)

    def trajectory(self, eps, n_steps, cp=None, obs_every=0, runaway_un=0.0):
        return cl_trajectory(self.h, eps, n_steps, cp, obs_every, runaway_un)

    def links(self):
        return cl_get_links(self.h, self.V)

    def set_links(self, U):
        cl_set_links(self.h, U)

    def drift(self):
        return cl_drift(self.h, self.V)

    def cool_gradient(self):
        return cl_cool_gradient(self.h, self.V)

    def qdensity(self):
        return cl_qdensity(self.h, self.V)

    @property
    def step_count(self):
        return cl_get_step(self.h)

    def launches(self):
        return cl_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            cl_free(self.h)
            self.h = None
        if getattr(self, "_own", None):
            cl_stream_destroy(self._own)
            self._own = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
