"""Bounded waits (cl_wait, cl_batch_wait): a caller that must not block on a
slow chain gets CL_ERR_TIMEOUT when the work outlasts its time limit, and the
work itself is unaffected -- waited for again it finishes, with the same
links as a chain that was never polled.  The slow work is just long (many
steps of a 16^4 lattice); nothing is made to hang."""
import numpy as np
import pytest

from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def _lat(seed=5):
    return cl.Lattice((16, 16, 16, 16), beta=6.0, theta=1.0, seed=seed, start=cl.CL_START_HOT, own_stream=True)


def test_wait_times_out_then_completes():
    cp = cl.make_cool(0.005, 1.0, cl.CL_D1, forced_sweeps=10)
    with _lat() as a, _lat() as b:
        for lat in (a, b):
            lat.trajectory(0.005, 40, cp)  # ~0.2 s of FP64 work queued
        assert cl.cl_wait(a.h, 0.0) is False  # a zero limit on running work
        assert cl.cl_wait(a.h, 1e-4) is False
        assert cl.cl_wait(a.h, 120.0) is True
        b.synchronize()
        assert np.array_equal(a.links(), b.links())
        assert cl.cl_wait(a.h, 0.0) is True  # nothing queued: done at once
    with pytest.raises(cl.CLError) as ei:
        cl.cl_wait(None, 1.0)
    assert ei.value.status == cl.CL_ERR_INVALID


def test_batch_wait_times_out_then_completes():
    lats = [_lat(seed=s) for s in (6, 7)]
    cp = cl.make_cool(0.005, 1.0, cl.CL_D1, forced_sweeps=10)
    try:
        with cl.Batch(lats, [0.005, 0.005], [cp, cp]) as b:
            b.run(40)
            assert cl.cl_batch_wait(b.h, 1e-4) is False
            assert cl.cl_batch_wait(b.h, 120.0) is True
            assert all(lat.step_count == 40 for lat in lats)
    finally:
        for lat in lats:
            lat.close()
