"""Checkpoint / resume: a lattice loaded from a checkpoint continues bit for
bit as the saved one does (counter-based noise, device step state, cooling
state and adaptive step size all in the checkpoint)."""
import numpy as np
import pytest

from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def _run(lat, cp, n):
    for _ in range(n):
        lat.step(0.01, 1)
        lat.cool(cp)


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE])
def test_resume_is_bit_for_bit(prec):
    L = (4, 6, 4, 4)
    cp = cl.make_cool(0.01, 0.5, cl.CL_D2_MEANABS, n_min=1, n_max=6, tol_rel=0.05)
    with cl.Lattice(L, beta=5.9, theta=1.5, prec=prec, seed=21, start=cl.CL_START_HOT, gauge_sigma=0.05,
                    own_stream=True) as a:
        a.set_adaptive_step(4.0)
        a.set_blocks([64, 32, 128, 256, 96])
        _run(a, cp, 4)
        ck = a.save_state()
        assert len(ck) == cl.cl_state_size(a.h)
        _run(a, cp, 4)
        ref = (a.links(), a.observables(), a.last_cool_report(), a.langevin_time(), a.step_count, a.blocks())
    # a lattice of the same shape but other parameters takes the checkpoint over
    with cl.Lattice(L, beta=6.3, theta=0.0, prec=prec, seed=99, own_stream=True) as b:
        b.load_state(ck)
        assert b.step_count == 4
        _run(b, cp, 4)
        got = (b.links(), b.observables(), b.last_cool_report(), b.langevin_time(), b.step_count, b.blocks())
    assert np.array_equal(got[0], ref[0])
    assert got[1:] == ref[1:]


def test_bad_checkpoints_are_refused():
    with cl.Lattice((4, 4, 4, 4), seed=1) as a, cl.Lattice((4, 4, 4, 6), seed=1) as b, \
            cl.Lattice((4, 4, 4, 4), prec=cl.CL_FP32_STORAGE, seed=1) as c:
        ck = a.save_state()
        for lat in (b, c):  # other extents, other precision
            with pytest.raises(cl.CLError) as ei:
                lat.load_state(ck)
            assert ei.value.status == cl.CL_ERR_INVALID
        with pytest.raises(cl.CLError):
            a.load_state(b"\0" * len(ck))  # not a checkpoint
        with pytest.raises(cl.CLError):
            a.load_state(ck[: len(ck) // 2])  # truncated
        a.load_state(ck)  # the good one still loads
