"""The request server: each request's result is the same alone and in the
mix (bit for bit: the chain's noise is keyed by its own seed, and its kernels
and reductions do not depend on its neighbours), admission respects the slot
count and the memory budget, idle lattices are reused, and a served FP64
trajectory agrees with the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


COOL = dict(alpha=1.0, mode=cl.CL_D2_MEANABS, n_min=1, n_max=6, tol_rel=0.02)


def _cool(eps):
    return cl.make_cool(eps, **COOL)


def _requests():
    specs = [((4, 4, 4, 4), 5.7, 0.0, 30), ((6, 6, 6, 6), 6.0, 1.0, 17), ((5, 4, 6, 3), 5.9, 0.5, 23),
             ((8, 8, 8, 8), 6.1, 2.0, 12), ((4, 4, 4, 4), 6.2, 1.5, 9), ((6, 6, 6, 6), 5.6, 0.3, 25),
             ((3, 5, 4, 4), 6.0, 1.0j, 14)]
    return [cl.make_request(L, b, th, 0.01, n, seed=100 + i, start=cl.CL_START_HOT, gauge_sigma=0.02, tag=i)
            for i, (L, b, th, n) in enumerate(specs)]


def _alone(req, prec):
    L = tuple(req.L)
    with cl.Lattice(L, beta=req.beta, theta=complex(req.theta_re, req.theta_im), prec=prec, seed=req.seed,
                    start=req.start, gauge_sigma=req.gauge_sigma) as lat:
        for _ in range(req.n_steps):
            lat.step(req.eps, 1)
            rep = lat.cool(_cool(req.eps))
        return lat.observables(), rep


def _serve(reqs, prec, **kw):
    cfg = dict(hbm_budget_bytes=4e9, max_slots=3, prec=prec, chunk_steps=4, use_graphs=True,
               cool=_cool(0.01), blocks_from_autotune=True)
    cfg.update(kw)
    with cl.Server(cl.make_server_config(**cfg)) as srv:
        for r in reqs:
            srv.submit(r)
        res = srv.drain(len(reqs))
        st = srv.stats()
    return {r["tag"]: r for r in res}, st


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE, cl.CL_DF64])
def test_each_result_same_alone_and_in_the_mix(prec):
    reqs = _requests()
    got, st = _serve(reqs, prec)
    assert st["completed"] == len(reqs) and st["peak_active"] <= 3 and st["pooled"] >= 1
    for r in reqs:
        obs, rep = _alone(r, prec)
        g = got[r.tag]
        assert g["status"] == cl.CL_OK and g["n_steps"] == r.n_steps
        assert g["obs"] == obs, r.tag
        assert g["last_cool"] == rep, r.tag
        assert g["t_submit"] <= g["t_admit"] <= g["t_done"]


def test_eager_server_equals_graph_server():
    reqs = _requests()[:4]
    a, _ = _serve(reqs, cl.CL_FP64, use_graphs=True, max_slots=4)
    b, _ = _serve(reqs, cl.CL_FP64, use_graphs=False, max_slots=1, blocks_from_autotune=False)
    for r in reqs:
        assert a[r.tag]["obs"] == b[r.tag]["obs"]


def test_memory_budget_bounds_the_resident_chains():
    one = cl.cl_lattice_bytes(cl.make_params((6, 6, 6, 6), prec=cl.CL_FP64))
    reqs = [cl.make_request((6, 6, 6, 6), 6.0, 1.0, 0.01, 6, seed=7 + i, tag=i) for i in range(5)]
    got, st = _serve(reqs, cl.CL_FP64, hbm_budget_bytes=2.5 * one, max_slots=8)
    assert st["completed"] == 5 and st["peak_active"] == 2
    assert st["peak_bytes"] <= 2.5 * one
    # a request larger than the whole budget is refused at submission
    with cl.Server(cl.make_server_config(hbm_budget_bytes=0.5 * one, prec=cl.CL_FP64)) as srv:
        with pytest.raises(cl.CLError) as ei:
            srv.submit(reqs[0])
        assert ei.value.status == cl.CL_ERR_INVALID
    # lattices of another shape evict idle ones to make room
    mixed = reqs[:2] + [cl.make_request((8, 6, 6, 6), 6.0, 1.0, 0.01, 4, seed=50, tag=9)]
    got, st = _serve(mixed, cl.CL_FP64, hbm_budget_bytes=2.2 * one, max_slots=1)
    assert st["completed"] == 3 and st["peak_bytes"] <= 2.2 * one
    assert got[9]["obs"] == _alone(mixed[2], cl.CL_FP64)[0]


def test_served_trajectory_against_the_oracle():
    L, beta, theta, eps, n = (4, 4, 4, 4), 6.0, 1.0, 0.01, 12
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D1, forced_sweeps=3)
    req = cl.make_request(L, beta, theta, eps, n, seed=11, start=cl.CL_START_COLD, gauge_sigma=0.05)
    cfg = cl.make_server_config(hbm_budget_bytes=1e9, max_slots=2, prec=cl.CL_FP64, chunk_steps=5,
                                cool=cl.make_cool(**cpar))
    with cl.Server(cfg) as srv:
        srv.submit(req)
        res = srv.drain(1)[0]
    U = O.random_gauge(L, O.cold_start(L), 11, 0.05)
    for step in range(n):
        U = O.cl_step(L, U, beta, theta, eps, 11, step)
        U, _ = O.cool(L, U, O.cool_params(**cpar))
    ref = O.observables(L, U, beta, theta)
    for k in ("plaq_re", "plaq_im", "un", "q_re", "q_im", "s_re", "s_im"):
        assert abs(res["obs"][k] - ref[k]) < 1e-11 * max(1.0, abs(ref[k])), k


def test_run_trace_returns_every_request():
    reqs = _requests()
    arrivals = np.linspace(0.0, 0.03, len(reqs))
    cfg = cl.make_server_config(hbm_budget_bytes=4e9, max_slots=4, prec=cl.CL_FP32_STORAGE, chunk_steps=4,
                                cool=_cool(0.01))
    with cl.Server(cfg) as srv:
        res = srv.run_trace(reqs, arrivals)
    assert sorted(r["tag"] for r in res) == list(range(len(reqs)))
    for r in res:
        assert r["t_done"] > r["t_submit"] and r["status"] == cl.CL_OK


def test_runaway_requests_stop_early():
    """A chain whose unitarity norm after a chunk exceeds the bound stops
    there with CL_ERR_RUNAWAY; its neighbour (theta = 0 from the cold start,
    which stays in SU(3) to rounding) runs to the end as if alone."""
    bad = cl.make_request((4, 4, 4, 4), 5.6, 2.0, 0.01, 400, seed=3, start=cl.CL_START_HOT, tag=0)
    good = cl.make_request((4, 4, 4, 4), 6.0, 0.0, 0.01, 20, seed=4, start=cl.CL_START_COLD, tag=1)
    cfg = cl.make_server_config(hbm_budget_bytes=1e9, max_slots=4, prec=cl.CL_FP64, chunk_steps=4,
                                cool=_cool(0.01), runaway_un=1.0 + 1e-9)
    with cl.Server(cfg) as srv:
        srv.submit(bad)
        srv.submit(good)
        res = {r["tag"]: r for r in srv.drain(2)}
        st = srv.stats()
    assert res[0]["status"] == cl.CL_ERR_RUNAWAY and 4 <= res[0]["n_steps"] <= 12
    assert res[1]["status"] == cl.CL_OK and res[1]["n_steps"] == 20
    assert res[1]["obs"] == _alone(good, cl.CL_FP64)[0]
    assert st["runaways"] == 1
