"""Host check of the exact fixed-point Laplacian numerator used by the FP64 residual
kernels (csrc/fixed_lap.cuh), compiled for the CPU and compared with exact rational
arithmetic (Python fractions):

* each value's fixed-point image is trunc(v * 2^(1080 - emax)), emax the largest biased
  exponent of the set;
* the integer numerator sum(neighbours) - 2D * centre is formed without overflow;
* its conversion to binary64 is the correctly rounded (nearest, ties to even) value;
* against the exact numerator of the unrounded values the error stays within the FP64
  evaluation's own bound (a few ulps of the largest value).
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2308_11469_gb300", "csrc")

PROBE = r"""
#include "fixed_lap.cuh"
#include <cmath>
#include <cstdio>
#include <random>
int main() {
    std::mt19937_64 g(12345);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    for (int t = 0; t < 20000; ++t) {
        const int D = 2 + (t & 1), nv = 2 * D + 1;
        double v[7];
        const int sc = (int)(g() % 600) - 300;
        const int spread = (t % 3 == 0) ? 70 : 3;
        for (int i = 0; i < nv; ++i) {
            v[i] = U(g) * std::ldexp(1.0, sc + (int)(g() % spread));
            if (g() % 40 == 0) v[i] = 0.0;
            if (t % 97 == 0 && i == 1) v[i] = -v[0];          // exact cancellation
        }
        int emax = 0;
        for (int i = 0; i < nv; ++i) emax = emax > helm::fx_exp(v[i]) ? emax : helm::fx_exp(v[i]);
        if (emax < helm::FX_EMIN || emax > helm::FX_EMAX) continue;
        long long F[7], S = 0;
        for (int i = 0; i < nv; ++i) F[i] = helm::fx_fix(v[i], emax);
        for (int i = 1; i < nv; ++i) S += F[i];
        const long long L = S - (long long)(2 * D) * F[0];
        const double r = helm::fx_to_double(L, emax);
        std::printf("%d %d", D, emax);
        for (int i = 0; i < nv; ++i) std::printf(" %a %lld", v[i], F[i]);
        std::printf(" %lld %a\n", L, r);
    }
    return 0;
}
"""


def _compile(tmp):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = os.path.join(tmp, "probe.cpp")
    exe = os.path.join(tmp, "probe")
    with open(src, "w") as fh:
        fh.write(PROBE)
    inc = ["-I", CSRC]
    cuda_inc = "/usr/local/cuda/include"
    if os.path.isdir(cuda_inc):
        inc += ["-I", cuda_inc]
    r = subprocess.run([cxx, "-std=c++17", "-O2", *inc, src, "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("fixed_lap.cuh does not build for the host here: " + r.stderr[-300:])
    return exe


def test_fixed_point_numerator_is_exact_and_correctly_rounded(tmp_path):
    exe = _compile(str(tmp_path))
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    assert len(out) > 15000
    worst = 0.0
    for line in out:
        p = line.split()
        D, emax = int(p[0]), int(p[1])
        nv = 2 * D + 1
        vals = [float.fromhex(p[2 + 2 * i]) for i in range(nv)]
        fix = [int(p[3 + 2 * i]) for i in range(nv)]
        L, r = int(p[2 + 2 * nv]), float.fromhex(p[3 + 2 * nv])
        scale = Fr(2) ** (1080 - emax)
        for v, F in zip(vals, fix):
            q = Fr(v) * scale
            assert F == (math.floor(q) if q >= 0 else -math.floor(-q))      # truncation
            assert abs(F) < 2 ** 58
        assert L == sum(fix[1:]) - 2 * D * fix[0]
        assert abs(L) < 2 ** 62
        exact_fixed = Fr(L) / scale
        assert r == float(exact_fixed)                # nearest binary64, ties to even
        exact = sum(Fr(v) for v in vals[1:]) - 2 * D * Fr(vals[0])
        big = max(abs(Fr(v)) for v in vals)
        worst = max(worst, float(abs(Fr(r) - exact) / big))
    # the truncations add below 2^-57 of the largest value each, the rounding half an ulp
    # of the result (at most 4 D times the largest): far inside the FP64 evaluation's bound
    assert worst <= 2.0 ** -49, worst
