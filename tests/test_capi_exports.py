"""The C-ABI library builds, loads and exports every function include/cl.h
declares; the binding declares the same names (no GPU needed, no compute)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "cl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cl_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("cl_init_lattice", "cl_step", "cl_cool", "cl_observables", "cl_trajectory",
              "cl_get_links", "cl_set_links", "cl_free", "cl_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1311_1056_gb300 import build, cl
    build.build()
    lib = cl.load()
    for n in declared_functions():
        assert hasattr(lib, n), n
        assert n in cl.SIGNATURES, n
    assert lib.cl_version() == 1
    assert lib.cl_status_str(cl.CL_ERR_NONFINITE) == b"non-finite links"


def test_invalid_arguments_fail_without_device_work():
    from paper_1311_1056_gb300 import cl
    p = cl.make_params((4, 0, 4, 4))
    with pytest.raises(cl.CLError) as e:
        cl.cl_init_lattice(p)
    assert e.value.status == cl.CL_ERR_INVALID
    assert "extent" in cl.cl_last_error()
    with pytest.raises(cl.CLError):
        cl.cl_step(None, 0.01, 1)
