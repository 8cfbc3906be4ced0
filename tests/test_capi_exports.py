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
    for args in ((7, 1, 0, 0, 0, 4), (cl.CL_DF64, 1, 0, 4, 0, 4), (cl.CL_FP64, 1, 0, 0, -1, 4),
                 (cl.CL_FP64, 1, 0, 0, 0, -2)):  # precision, direction, site range
        with pytest.raises(cl.CLError) as e:
            cl.noise_sample(*args)
        assert e.value.status == cl.CL_ERR_INVALID


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets
    the C compiler gives the header's structs."""
    import ctypes
    import shutil
    import subprocess
    from paper_1311_1056_gb300 import cl
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = ["cl_params", "cl_cool_params", "cl_obs", "cl_cool_report", "cl_request",
               "cl_server_config", "cl_result", "cl_server_stats"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cl.h"', "int main(void) {"]
    for s in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in getattr(cl, s)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().split("\n") if l)
    for s in structs:
        T = getattr(cl, s)
        assert int(got[s]) == ctypes.sizeof(T), s
        for f, _ in T._fields_:
            assert int(got["%s.%s" % (s, f)]) == getattr(T, f).offset, (s, f)


def test_oversized_lattice_is_rejected_before_any_device_work():
    """The largest lattice accepted has V * 54 <= 2^31 - 1 sites (79^4 =
    38.9 M); 80^4 is refused with CL_ERR_INVALID before any CUDA call."""
    from paper_1311_1056_gb300 import cl
    with pytest.raises(cl.CLError) as e:
        cl.cl_init_lattice(cl.make_params((80, 80, 80, 80)))
    assert e.value.status == cl.CL_ERR_INVALID and "too large" in cl.cl_last_error()
    p = cl.make_params((80, 80, 80, 80))
    with pytest.raises(cl.CLError):
        cl.cl_lattice_bytes(p)
    b64 = cl.cl_lattice_bytes(cl.make_params((79, 79, 79, 79)))
    b32 = cl.cl_lattice_bytes(cl.make_params((79, 79, 79, 79), prec=cl.CL_FP32_STORAGE))
    assert b64 > 280e9  # 54 FP64 matrices per site: more than one GB300 holds
    # FP32 storage: 50 matrices of half the size (no inverse field)
    assert abs(b32 / b64 - 50 / 108) < 1e-3
