"""The compile-time twiddle factors of the one-thread-per-line plane pass
(csrc/ct_trig.hpp) against the C library's cos/sin: a small host program is
compiled with g++ and its values compared to a 40-digit mpmath evaluation:
every value within 2 ulp of 1 of the exact one (a wrong series term or
quadrant would be off by orders of magnitude more)."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2505_02319_gb300", "csrc", "ct_trig.hpp")

PROG = r"""
#include <cstdio>
#include "ct_trig.hpp"
static_assert(ikr::CtTwiddle<48, 12>::c == 0.0, "quarter turn is exact");
int main() {
  const int ns[] = {2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 96, 7, 9, 1000};
  for (int n : ns)
    for (int k = -n; k <= 2 * n; ++k) {
      const ikr::CtCosSin v = ikr::ct_cossin(k, n);
      std::printf("%d %d %.17e %.17e\n", n, k, v.c, v.s);
    }
  return 0;
}
"""


@pytest.fixture(scope="module")
def values():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        with open(src, "w") as f:
            f.write(PROG)
        exe = os.path.join(d, "t")
        subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.dirname(os.path.abspath(HDR)), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return np.array([[float(t) for t in line.split()] for line in out.splitlines()])


def test_twiddles_match_library(values):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    err = 0.0
    for n, k, c, s in values:
        t = 2 * mpmath.pi * mpmath.mpf(int(k) % int(n)) / int(n)
        err = max(err, abs(float(mpmath.cos(t) - c)), abs(float(mpmath.sin(t) - s)))
    assert err <= 2.0 ** -51


def test_twiddles_are_exact_on_the_axes(values):
    n, k, c, s = values.T
    quarter = np.mod(4 * k, n) == 0
    assert np.all(np.isin(c[quarter], [-1.0, 0.0, 1.0])) and np.all(np.isin(s[quarter], [-1.0, 0.0, 1.0]))
    assert np.all(np.abs(c ** 2 + s ** 2 - 1) < 1.2e-15)
