"""The CL noise as each form's kernels draw it (cl_noise_sample) against the
oracle's Philox4x32-10 + Box-Muller normals (Sec. 2 noise; the counter
layout of the update): FP64 to rounding, DF64 (ln, sqrt and sincospi in
double-float) to 1e-13 relative, FP32 storage to float precision.  4M links
per form: the smallest radius uniform among them (~1e-7) reaches far into
the Gaussian tail, and the angles cover every quadrant boundary."""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu

N = 1 << 22


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


@pytest.fixture(scope="module")
def ref():
    return O.normals_sites(20240601, 7, 1000, N, 2, 0, 4)


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-14), (cl.CL_DF64, 1e-13)])
def test_noise_matches_oracle(ref, prec, tol):
    got = cl.noise_sample(prec, 20240601, 7, 2, 1000, N)
    assert np.abs(ref).max() > 5.0  # the sample reaches the tail
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() < tol, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_fp32_noise_at_float_precision(ref):
    got = cl.noise_sample(cl.CL_FP32_STORAGE, 20240601, 7, 2, 1000, N)
    err = np.abs(got - ref)
    assert np.quantile(err, 0.999) < 2e-6
    assert err.max() < 1e-3  # radius uniforms within 2^-25 of 1 (float spacing)


def test_noise_sample_edges():
    a = cl.noise_sample(cl.CL_DF64, 1, 0, 0, 0, 3)
    b = cl.noise_sample(cl.CL_DF64, 1, 0, 0, 1, 2)
    assert np.array_equal(a[1:], b)  # a link's numbers do not depend on the range
    assert cl.noise_sample(cl.CL_FP64, 1, 0, 0, 5, 0).shape == (0, 8)
