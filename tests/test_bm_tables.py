"""The FP64 noise's tables (paper_1311_1056_gb300/csrc/bm_tables.cuh) are
the output of their generator, and the values in them are what their
definitions say: ln(j/128), 1/(j/128), sin and cos(pi j/64), ln 2 split into
a 42-bit head and a tail, and the Taylor coefficients of sin and cos(pi y),
each checked against Python's math library to an ulp (no GPU needed)."""
import math
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1311_1056_gb300", "csrc")


def _header():
    with open(os.path.join(CSRC, "bm_tables.cuh")) as fh:
        return fh.read()


def _pairs(src, name):
    body = src.split(name)[1].split("};")[0]
    return [(float.fromhex(a), float.fromhex(b)) for a, b in re.findall(r"\{(\S+), (\S+)\},", body)]


def test_header_is_the_generator_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "bm_tables.py")], capture_output=True, text=True,
                         check=True).stdout
    assert out.strip() == _header().strip()


def test_table_values_match_their_definitions():
    src = _header()
    ln = _pairs(src, "BM_LN_TAB")
    assert len(ln) == 92
    for j, (rcp, lnc) in zip(range(90, 182), ln):
        c = j / 128
        assert abs(rcp - 1 / c) <= math.ulp(1 / c)
        assert abs(lnc - math.log(c)) <= math.ulp(math.log(c)) + 1e-300
    sc = _pairs(src, "BM_SC_TAB")
    assert len(sc) == 129
    for j, (s, c) in enumerate(sc):
        # reference on the first quadrant (the rounded angle pi m / 64 <= pi / 2
        # is off by at most 2e-16), carried to quadrant q by the symmetries
        q, m = divmod(j, 32)
        s1, c1 = math.sin(math.pi * m / 64), math.cos(math.pi * m / 64)
        rs, rc = [(s1, c1), (c1, -s1), (-s1, -c1), (-c1, s1), (s1, c1)][q]
        assert abs(s - rs) < 3e-16 and abs(c - rc) < 3e-16, (j, s, rs, c, rc)
        if j % 32 == 0:  # exact zeros and ones at multiples of pi/2
            assert {abs(s), abs(c)} == {0.0, 1.0}
    consts = {k: float.fromhex(v) for k, v in re.findall(r"const double (BM_\w+) = (\S+);", src)}
    hi, lo = consts["BM_LN2_HI"], consts["BM_LN2_LO"]
    assert abs(hi + lo - math.log(2)) <= math.ulp(math.log(2))
    assert hi == math.ldexp(round(math.ldexp(hi, 41)), -41)  # 42 significant bits: e * hi exact for |e| <= 53
    for k in (1, 3, 5, 7):
        want = (-1) ** (k // 2) * math.pi ** k / math.factorial(k)
        assert abs(consts["BM_S%d" % k] - want) <= 4 * math.ulp(want)
    for k in (2, 4, 6, 8):
        want = (-1) ** (k // 2) * math.pi ** k / math.factorial(k)
        assert abs(consts["BM_C%d" % k] - want) <= 4 * math.ulp(want)
