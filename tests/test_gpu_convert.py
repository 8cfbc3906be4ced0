"""The FP32-storage kernels widen floats to FP64 and narrow FP64 results to
float with integer operations (IEEE-754 field moves, round to nearest even)
instead of the hardware conversions, which issue on the narrow FP64 pipe.
The library's self-test compares both directions with the hardware
conversions bit for bit on 2^25 generated cases: every float bit pattern
class (normals, zeros, subnormals, infinities, NaNs) and doubles across the
whole float range, its underflow and overflow ends, with exact rounding ties."""
import pytest

from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


def test_integer_pipe_conversions_are_bit_exact():
    build.build()
    cl.load()
    for seed in (1, 0x9E3779B97F4A7C15):
        bad_f2d, bad_d2f = cl.cl_selftest_convert(seed, 1 << 25)
        assert bad_f2d == 0 and bad_d2f == 0, (seed, bad_f2d, bad_d2f)
