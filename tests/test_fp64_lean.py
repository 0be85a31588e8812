"""The few-FP64-instruction reciprocal and reciprocal square root used by the
SPAI kernels (csrc/fp64_lean.cuh), compiled as host C++ with the FP32 seed
exact and perturbed by +-2^-21, checked against long-double references:
every result within one ulp of the exact value.  CPU only (needs g++)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1606_01216_gb300", "csrc")

MAIN = r'''
#include "fp64_lean.cuh"
#include <cmath>
#include <cstdio>
#include <random>
using namespace airga::lean;
static double ulp(double x) { return std::nextafter(std::fabs(x), INFINITY) - std::fabs(x); }
int main() {
    std::mt19937_64 g(7);
    long bad = 0;
    double worst_r = 0, worst_s = 0;
    for (long k = 0; k < 3000000; ++k) {
        const int e = (int)(g() % 2000) - 1000;
        const double m = 1.0 + (double)(g() >> 11) * 0x1p-53;
        const double d = std::ldexp(m, e);
        const long double rr = 1.0L / (long double)d;
        const long double rs = 1.0L / std::sqrt((long double)d);
        const double er = (double)std::fabs((long double)rcp(d) - rr) / ulp((double)rr);
        const double es = (double)std::fabs((long double)rsqrt(d) - rs) / ulp((double)rs);
        if (er > worst_r) worst_r = er;
        if (es > worst_s) worst_s = es;
        if (er > 1.0 || es > 1.0) { if (bad < 5) std::printf("d=%a rcp %.3f ulp rsqrt %.3f ulp\n", d, er, es); ++bad; }
    }
    const double sp[] = {1.0, 2.0, 4.0, 0.5, 3.0, 0x1.fffffffffffffp0, 0x1p-1000, 0x1p1000, 1e-300, 1e300, 7.0e15, 0.1};
    for (double d : sp) {
        const double er = (double)std::fabs((long double)rcp(d) - 1.0L / d) / ulp(1.0 / d);
        const double es = (double)std::fabs((long double)rsqrt(d) - 1.0L / std::sqrt((long double)d)) / ulp(1.0 / std::sqrt(d));
        if (er > 1.0 || es > 1.0) { std::printf("special d=%a rcp %.3f rsqrt %.3f\n", d, er, es); ++bad; }
    }
    if (rcp(0.0) != 0.0 || rsqrt(0.0) != 0.0) { std::printf("zero\n"); ++bad; }
    if (neg_sign_of(2.0, 3.0) != -2.0 || neg_sign_of(2.0, -3.0) != 2.0 || neg_sign_of(2.0, 0.0) != -2.0) { std::printf("sign\n"); ++bad; }
    if (abs_of(-2.5) != 2.5 || abs_of(2.5) != 2.5) { std::printf("abs\n"); ++bad; }
    std::printf("worst rcp %.3f ulp, rsqrt %.3f ulp, bad %ld\n", worst_r, worst_s, bad);
    return bad != 0;
}
'''


@pytest.mark.parametrize("seed_scale", ["1.0", "(1.0 + 0x1p-21)", "(1.0 - 0x1p-21)"])
def test_lean_rcp_rsqrt_within_one_ulp(seed_scale):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "lean.cpp")
        exe = os.path.join(d, "lean")
        with open(src, "w") as f:
            f.write(MAIN)
        subprocess.check_call([gxx, "-std=c++17", "-O2", "-ffp-contract=off",
                               "-DAIRGA_LEAN_SEED_SCALE=" + seed_scale, "-I", CSRC, "-o", exe, src])
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "bad 0" in out.stdout, out.stdout
