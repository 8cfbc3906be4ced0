"""The FP64 noise (Sec. 2: real Gaussian noise by Box-Muller from the
Philox uniforms) takes ln and sincospi from tables at a grid of 1/128 and
1/64 and short polynomials in the remainder, since GB300's narrow FP64 pipe
made CUDA's general log and sincospi most of the noise's cost.  The library's
self-test compares both with CUDA's functions over 2^24 uniforms of the form
the noise uses, (k + 1/2) 2^-52: across the whole range, deep in the tail of
ln (k down to 0), next to 1, and next to the sine table's grid points.  The
end-to-end check against the oracle's normals is test_gpu_noise.py."""
import pytest

from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


def test_table_driven_ln_and_sincospi_within_a_few_ulp():
    build.build()
    cl.load()
    for seed in (3, 0xC0FFEE):
        ulp_ln, ulp_sc = cl.cl_selftest_box_muller(seed, 1 << 24)
        assert ulp_ln <= 2 and ulp_sc <= 3, (seed, ulp_ln, ulp_sc)
