"""The allocation-free observables entry point (cl_observables_noalloc).

Some callers cannot let a library allocate device memory: programs whose
device memory belongs to their own pool or arena, and latency-critical loops
that cannot afford cudaMalloc/cudaFree (which may synchronise the device).
For them cl_observables_noalloc reads caller-owned device links and writes
caller-owned device output, keeping its partial sums in a fixed array inside
the library.  This test (collected last on purpose) calls it through the
C-ABI several times in a row -- each call on a smaller lattice than the one
before, so the shared array still holds records of the previous call -- and
compares each result with the allocating entry point cl_observables.  The
first lattice, 24^4 (331,776 sites), needs more than CL_NOALLOC_MAX_BLOCKS
blocks of 128 threads, so its threads each sum several sites and the final
reduction reads all 2048 records; the last has a single block.  The small
lattice is also compared with the FP64 oracle directly.  The test allocates
the caller's buffers itself (with torch), as such a caller would with its own
allocator.
"""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu

CASES = [
    dict(L=(24, 24, 24, 24), beta=6.2, theta=1.0, seed=2, gauge_sigma=0.05),
    dict(L=(6, 4, 8, 5), beta=6.0, theta=1.0 + 0.2j, seed=3, gauge_sigma=0.08),
    dict(L=(3, 4, 2, 4), beta=5.7, theta=0.5j, seed=4, gauge_sigma=0.2),
]


def test_noalloc_observables_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    build.build()
    cl.load()
    for c in CASES:
        V = int(np.prod(c["L"]))
        with cl.Lattice(c["L"], beta=c["beta"], theta=c["theta"], seed=c["seed"],
                        start=cl.CL_START_HOT, gauge_sigma=c["gauge_sigma"]) as lat:
            lat.step(0.01, 2)  # a complex-Langevin state away from SU(3)
            ref = lat.observables()
            links = torch.empty(V * 4 * 18, dtype=torch.float64, device="cuda")
            cl.cl_get_links_device(lat.h, links.data_ptr())
            cl.cl_synchronize(lat.h)
        out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        cl.cl_observables_noalloc(links.data_ptr(), c["L"], c["beta"], c["theta"], out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = dict(zip([n for n, _ in cl.cl_obs._fields_], out.cpu().tolist()))
        for k, v in ref.items():
            tol = 1e-12 * max(1.0, abs(v)) if k != "max_det_dev" else 1e-14
            assert abs(got[k] - v) <= tol, (c["L"], k, got[k], v)
        if V <= 1000:  # the oracle's brute-force q_L is quick here
            U = links.cpu().numpy().view(np.complex128).reshape(V, 4, 3, 3)
            want = O.observables(c["L"], U, c["beta"], c["theta"])
            for k, v in want.items():
                tol = 1e-12 * max(1.0, abs(v)) if k != "max_det_dev" else 1e-14
                assert abs(got[k] - v) <= tol, ("oracle", c["L"], k, got[k], v)


def test_noalloc_flags_nonfinite_links():
    """A NaN entry in the caller's links turns max |det U - 1| into NaN."""
    torch = pytest.importorskip("torch")
    cl.load()
    L = (2, 3, 2, 2)
    V = int(np.prod(L))
    U = np.zeros((V, 4, 3, 3), complex)
    U[:] = np.eye(3)
    links = torch.from_numpy(U.view(np.float64).ravel().copy()).cuda()
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    cl.cl_observables_noalloc(links.data_ptr(), L, 6.0, 0.0, out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert out[9].item() == 0.0 and out[2].item() == 1.0
    links[5 * 18 + 3] = float("nan")
    cl.cl_observables_noalloc(links.data_ptr(), L, 6.0, 0.0, out.data_ptr(), 0)
    torch.cuda.synchronize()
    assert np.isnan(out[9].item())


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    cl.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(cl.CLError) as e:
        cl.cl_observables_noalloc(buf.data_ptr(), (4, 0, 4, 4), 6.0, 0.0, buf.data_ptr(), 0)
    assert e.value.status == cl.CL_ERR_INVALID
    with pytest.raises(cl.CLError) as e:
        cl.cl_observables_noalloc(buf.data_ptr(), (1024, 1024, 1024, 2), 6.0, 0.0, buf.data_ptr(), 0)
    assert e.value.status == cl.CL_ERR_INVALID
    assert "CL_NOALLOC_MAX_SITES" in cl.cl_last_error()
