"""The integer-only IEEE conversions used by the learned-SPAI kernels
(csrc/ieee_conv.cuh), compiled as host C++ and checked bit for bit against
the host's IEEE-754 conversions on random, range-targeted and special
inputs.  CPU only (needs g++)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1606_01216_gb300", "csrc")

MAIN = r'''
#include "ieee_conv.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
using namespace airga::ieee;
static unsigned fu(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float uf(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static unsigned long long du(double d) { unsigned long long u; std::memcpy(&u, &d, 8); return u; }
static double ud(unsigned long long u) { double d; std::memcpy(&d, &u, 8); return d; }
static bool same_f(float a, float b) { return std::isnan(a) ? std::isnan(b) : fu(a) == fu(b); }
static bool same_d(double a, double b) { return std::isnan(a) ? std::isnan(b) : du(a) == du(b); }
int main() {
    std::mt19937_64 g(12345);
    long bad = 0;
    for (long k = 0; k < 4000000; ++k) {
        unsigned long long bits = g();
        if (k % 4 == 1)        // binary32 normal range
            bits = (bits & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(1023 - 126 + (g() % 252)) << 52);
        else if (k % 4 == 2)   // around and below the binary32 subnormal range
            bits = (bits & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(1023 - 152 + (g() % 28)) << 52);
        const double x = ud(bits);
        if (!same_f((float)x, f64_to_f32(x))) { if (bad < 5) std::printf("f64_to_f32 %a\n", x); ++bad; }
        if (!same_d(x / 2.0, half_of(x))) { if (bad < 5) std::printf("half_of %a\n", x); ++bad; }
        const float f = uf((unsigned)g());
        if (!same_d((double)f, f32_to_f64(f))) { if (bad < 5) std::printf("f32_to_f64 %a\n", f); ++bad; }
    }
    const double sp[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 1e-310, -1e-310, 4.9e-324,
                         2.2250738585072014e-308, 4.450147717014403e-308, 3.4028235677973366e38,
                         3.4028234663852886e38, 1e39, 1.17549435e-38, 1.1754942e-38, 1.4e-45,
                         7.0e-46, 0.1, -7.5, 1.0 + 1.0 / (1 << 24), 1.0 + 3.0 / (1 << 24)};
    for (double x : sp) {
        if (!same_f((float)x, f64_to_f32(x))) { std::printf("special f64_to_f32 %a\n", x); ++bad; }
        if (!same_d(x / 2.0, half_of(x))) { std::printf("special half_of %a\n", x); ++bad; }
        const float f = (float)x;
        if (!same_d((double)f, f32_to_f64(f))) { std::printf("special f32_to_f64 %a\n", f); ++bad; }
    }
    std::printf("bad %ld\n", bad);
    return bad != 0;
}
'''


def test_integer_ieee_conversions_match_host():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "conv.cpp")
        exe = os.path.join(d, "conv")
        with open(src, "w") as f:
            f.write(MAIN)
        subprocess.check_call([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, "-o", exe, src])
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "bad 0" in out.stdout
