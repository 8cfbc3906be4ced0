"""The device-side adaptive cooling rule against the exact one-link model.

The one-link model of Sec. 3 (`one_link_model.py`) fixes, in closed form, the
sweep at which every branch of the sweep-count rule stops (floor, progress,
n_min, n_max, the D < d_guard skip) for D_0, D_1 and D_2 (RMS).  Here the same
cases run through the C-ABI's cl_cool, whose rule is decided on the device;
the count, the unitarity norm before and after and the last alpha_ad must
match the closed form (FP64 and double-float forms; links of the FP32-storage
form carry rounding far above what separates a count from its neighbour at
the tighter cases, so that form is checked on the cases whose margin allows).
"""
import pytest

import one_link_model as M
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu

L1 = (1, 1, 1, 1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_DF64, cl.CL_FP32_STORAGE], ids=["fp64", "df64", "fp32"])
@pytest.mark.parametrize("case", M.CASES, ids=[c[0] for c in M.CASES])
def test_device_rule_count(case, prec):
    _name, d0, c, eps, alpha, mode, n_min, n_max, tol, d_floor = case
    # the FP32-storage form skips cooling below D = 1e-6 (its links' rounding)
    guard = 1e-6 if prec == cl.CL_FP32_STORAGE else 1e-12
    P = M.predict(d0, c, eps, alpha, mode, n_min, n_max, tol, d_floor, guard)
    if prec == cl.CL_FP32_STORAGE and P["margin"] < 1e-2:
        pytest.skip("count margin below the FP32 storage rounding of the norm's differences")
    with cl.Lattice(L1, prec=prec) as lat:
        lat.set_links(M.lattice(d0, c))
        rep = lat.cool(cl.make_cool(eps, alpha, mode, n_min, n_max, tol, d_floor, guard))
    tol_un = {cl.CL_FP64: 1e-13, cl.CL_DF64: 1e-12, cl.CL_FP32_STORAGE: 1e-5}[prec]
    assert rep["sweeps"] == P["sweeps"]
    assert abs(rep["un_before"] - P["un_before"]) < tol_un
    assert abs(rep["un_after"] - P["un_after"]) < tol_un
    tol_a = 1e-10 if prec != cl.CL_FP32_STORAGE else 1e-3
    assert abs(rep["alpha_ad_last"] - P["alpha_ad_last"]) <= tol_a * max(1.0, P["alpha_ad_last"])
