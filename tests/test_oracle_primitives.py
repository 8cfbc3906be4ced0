"""Pins of the oracle's building blocks against library routines and
published reference values (no GPU).

* Philox4x32-10: the known-answer vectors published with the generator
  (Salmon, Moraes, Dror, Shaw, SC'11, Random123 distribution) and an
  independent implementation (ATen's header-only Philox engine), compiled here.
* exp, inverse, det: scipy.linalg.expm, numpy.linalg.inv, numpy.linalg.det.
* Gell-Mann matrices: Hermitian, traceless, Tr l_a l_b = 2 delta_ab and the
  su(2) subalgebra [l_1, l_2] = 2i l_3.
* Box-Muller normals: moments of a large sample.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.linalg

import oracle as O
import lattice_inputs as LI

# Known-answer vectors of Philox4x32-10: (counter, key) -> output.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(ctr, key, expect):
    assert tuple(O.philox(ctr, key)) == expect


ATEN_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  for (int t = 1; t + 5 < argc; t += 6) {
    unsigned c[4], k[2];
    for (int i = 0; i < 4; ++i) c[i] = strtoul(argv[t + i], 0, 0);
    for (int i = 0; i < 2; ++i) k[i] = strtoul(argv[t + 4 + i], 0, 0);
    uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
    at::Philox4_32 e(seed, (uint64_t)c[2] | ((uint64_t)c[3] << 32),
                     (uint64_t)c[0] | ((uint64_t)c[1] << 32));
    for (int i = 0; i < 4; ++i) printf("%u ", e());
    printf("\n");
  }
}
"""


def test_philox_matches_independent_implementation():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen Philox header not available")
    r = LI.rng(5)
    cases = [tuple(int(v) for v in r.integers(0, 2**32, size=6)) for _ in range(64)]
    cases += [(7, 3, 2 | (1 << 8), 1, 1, 0), (1023, 999, 3, 0, 0xdeadbeef, 0x12345678)]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        with open(src, "w") as fh:
            fh.write(ATEN_PROG)
        try:
            subprocess.run(["g++", "-std=c++17", "-O1", "-I" + inc, src, "-o", exe], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError as e:
            pytest.skip("cannot compile the ATen Philox engine: %s" % e.stderr[:200])
        out = subprocess.run([exe] + [str(v) for c in cases for v in c], check=True,
                             capture_output=True, text=True).stdout.split("\n")
    for c, line in zip(cases, out):
        ref = [int(v) for v in line.split()]
        assert O.philox(c[:4], c[4:]) == ref, c


def test_normals_moments():
    g = np.concatenate([O.normals(11, step, site, mu, 0, 4)
                        for step in range(3) for site in range(700) for mu in range(4)])
    n = g.size  # 67200
    assert abs(g.mean()) < 4.0 / np.sqrt(n)
    assert abs(g.var() - 1.0) < 4.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(g**4) - 3.0) < 4.0 * np.sqrt(96.0 / n)
    # pairs from one counter are uncorrelated
    assert abs(np.mean(g[0::2] * g[1::2])) < 4.0 / np.sqrt(n / 2)


def test_normals_streams_differ():
    a = O.normals(1, 0, 5, 1, 0, 4)
    assert not np.allclose(a, O.normals(1, 1, 5, 1, 0, 4))   # step
    assert not np.allclose(a, O.normals(1, 0, 6, 1, 0, 4))   # site
    assert not np.allclose(a, O.normals(1, 0, 5, 2, 0, 4))   # mu
    assert not np.allclose(a, O.normals(1, 0, 5, 1, 1, 4))   # stream
    assert not np.allclose(a, O.normals(2, 0, 5, 1, 0, 4))   # seed
    np.testing.assert_array_equal(a, O.normals(1, 0, 5, 1, 0, 4))


def test_gellmann_algebra():
    lam = [O.gellmann(a) for a in range(1, 9)]
    for a in range(8):
        np.testing.assert_allclose(lam[a], lam[a].conj().T, atol=0)
        assert abs(np.trace(lam[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2.0 * (a == b)) < 1e-14
    np.testing.assert_allclose(lam[0] @ lam[1] - lam[1] @ lam[0], 2j * lam[2], atol=1e-15)
    # completeness: sum_a Tr(l_a X) l_a = 2 (X - Tr X / 3)
    X = LI.random_sl3c(LI.rng(1), 1)[0]
    S = sum(np.trace(l @ X) * l for l in lam)
    np.testing.assert_allclose(S, 2 * (X - np.trace(X) / 3 * np.eye(3)), atol=1e-14)


@pytest.mark.parametrize("scale", [1e-3, 0.3, 2.0, 7.0])
def test_expm_matches_scipy(scale):
    r = LI.rng(int(scale * 100))
    for _ in range(20):
        A = scale * (r.normal(size=(3, 3)) + 1j * r.normal(size=(3, 3)))
        ref = scipy.linalg.expm(A)
        np.testing.assert_allclose(O.expm(A), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_inverse_and_det_match_numpy():
    r = LI.rng(3)
    for _ in range(50):
        A = r.normal(size=(3, 3)) + 1j * r.normal(size=(3, 3))
        np.testing.assert_allclose(O.inverse(A), np.linalg.inv(A), atol=1e-12)
        assert abs(O.det(A) - np.linalg.det(A)) < 1e-12
