// FP64 reciprocal and reciprocal square root that spend few FP64-pipe
// instructions.  On GB300 the FP64 pipe executes 2 operations per clock per
// SM; the SPAI kernels are bound by it, so every FP64 instruction counts.
//
// Method: range reduction and sign handling with integer operations, a seed
// from the FP32 hardware approximation (rcp / rsqrt of the reduced argument,
// relative error below 2^-21 including the truncation of the argument to
// FP32), then two Newton-Raphson steps in FP64:
//   reciprocal:   y <- y + y (1 - d y)                  (2 FMA per step)
//   rsqrt:        y <- y + y (1/2 - (d/2) y^2)          (1 MUL + 2 FMA per step)
// Each step squares the relative error (Newton-Raphson is quadratically
// convergent), so two steps take 2^-21 to below 2^-84 before the final
// rounding: the results are within one ulp of the correctly rounded value
// (checked against the host on random and targeted inputs, with the seed
// perturbed by 2^-21 both ways).  Arguments must be positive normal numbers
// in [2^-1021, 2^1021]; 0 gives 0 (callers treat a zero pivot as rank
// deficiency), other inputs are outside the contract.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define AIRGA_LEAN __device__ __forceinline__
#else
#include <cmath>
#include <cstring>
#define AIRGA_LEAN inline
#ifndef AIRGA_LEAN_SEED_SCALE
#define AIRGA_LEAN_SEED_SCALE 1.0   // host tests perturb the seed by up to 2^-21
#endif
#endif

namespace airga {
namespace lean {

// FP32 seeds: the hardware approximations (PTX rcp.approx / rsqrt.approx,
// relative error about 2^-23) on the GPU; on the host (tests) the libm value
// scaled by AIRGA_LEAN_SEED_SCALE to emulate a seed error.
AIRGA_LEAN float rcp_seed(float x) {
#if defined(__CUDACC__)
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return (float)((1.0 / (double)x) * AIRGA_LEAN_SEED_SCALE);
#endif
}

AIRGA_LEAN float rsqrt_seed(float x) {
#if defined(__CUDACC__)
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return (float)((1.0 / std::sqrt((double)x)) * AIRGA_LEAN_SEED_SCALE);
#endif
}

AIRGA_LEAN unsigned long long bits_of(double x) {
#if defined(__CUDACC__)
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}

AIRGA_LEAN double from_bits(unsigned long long u) {
#if defined(__CUDACC__)
    return __longlong_as_double((long long)u);
#else
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}

AIRGA_LEAN float f_from_bits(unsigned u) {
#if defined(__CUDACC__)
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

AIRGA_LEAN unsigned f_bits(float f) {
#if defined(__CUDACC__)
    return __float_as_uint(f);
#else
    unsigned u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}

// FP32 value of a double whose exponent field is 1023 or 1024 (value in
// [1, 4)), by truncating the fraction (a seed needs no rounding)
AIRGA_LEAN float reduced_to_f32(unsigned long long b) {
    const unsigned ex = (unsigned)(b >> 52) & 0x7FFu;              // 1023 or 1024
    const unsigned frac = (unsigned)(b >> 29) & 0x7FFFFFu;         // top 23 fraction bits
    return f_from_bits(((ex - 1023u + 127u) << 23) | frac);
}

// 1/d for positive normal d (0 -> 0)
AIRGA_LEAN double rcp(double d) {
    const unsigned long long b = bits_of(d);
    if (b == 0ull) return 0.0;
    const int e = (int)((b >> 52) & 0x7FFu) - 1023;                // d = m 2^e, m in [1, 2)
    const double m = from_bits((b & 0x000FFFFFFFFFFFFFull) | (1023ull << 52));
    const float yf = rcp_seed(reduced_to_f32(bits_of(m)));          // ~1/m in (1/2, 1]
    // seed as a double: exact widening of the FP32 bits
    const unsigned yb = f_bits(yf);
    double y = from_bits(((unsigned long long)(((yb >> 23) & 0xFFu) - 127u + 1023u) << 52) |
                         ((unsigned long long)(yb & 0x7FFFFFu) << 29));
    double t = fma(-m, y, 1.0);
    y = fma(y, t, y);
    t = fma(-m, y, 1.0);
    y = fma(y, t, y);                                               // 1/m, y in (1/2, 1]
    // 1/d = (1/m) 2^-e: adjust the exponent field
    const unsigned long long yb2 = bits_of(y);
    return from_bits(yb2 - ((unsigned long long)(long long)e << 52));
}

// 1/sqrt(d) for positive normal d (0 -> 0)
AIRGA_LEAN double rsqrt(double d) {
    const unsigned long long b = bits_of(d);
    if (b == 0ull) return 0.0;
    const int E = (int)((b >> 52) & 0x7FFu) - 1023;
    const int k = E >> 1;                                           // floor(E / 2)
    const int r = E - 2 * k;                                        // 0 or 1
    // m = d 2^(-2k) in [1, 4)
    const double m = from_bits((b & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(1023 + r) << 52));
    const float yf = rsqrt_seed(reduced_to_f32(bits_of(m)));        // ~1/sqrt(m) in (1/2, 1]
    const unsigned yb = f_bits(yf);
    double y = from_bits(((unsigned long long)(((yb >> 23) & 0xFFu) - 127u + 1023u) << 52) |
                         ((unsigned long long)(yb & 0x7FFFFFu) << 29));
    const double h = from_bits(bits_of(m) - (1ull << 52));         // m / 2, exact
    double hy = h * y;
    double t = fma(-hy, y, 0.5);
    y = fma(y, t, y);
    hy = h * y;
    t = fma(-hy, y, 0.5);
    y = fma(y, t, y);                                               // 1/sqrt(m)
    // 1/sqrt(d) = (1/sqrt(m)) 2^-k
    return from_bits(bits_of(y) - ((unsigned long long)(long long)k << 52));
}

// One-Newton-step variants: relative error below 2^-43 (the seed's ~2^-22
// squared, plus rounding) for two FP64 instructions fewer (rcp) / three fewer
// (rsqrt).  Enough wherever the result only has to be accurate far beyond the
// method's tolerances (the Householder scalars of the SPAI least squares,
// whose solution is checked to 1e-10).
AIRGA_LEAN double rcp1(double d) {
    const unsigned long long b = bits_of(d);
    if (b == 0ull) return 0.0;
    const int e = (int)((b >> 52) & 0x7FFu) - 1023;
    const double m = from_bits((b & 0x000FFFFFFFFFFFFFull) | (1023ull << 52));
    const unsigned yb = f_bits(rcp_seed(reduced_to_f32(bits_of(m))));
    double y = from_bits(((unsigned long long)(((yb >> 23) & 0xFFu) - 127u + 1023u) << 52) |
                         ((unsigned long long)(yb & 0x7FFFFFu) << 29));
    y = fma(y, fma(-m, y, 1.0), y);
    return from_bits(bits_of(y) - ((unsigned long long)(long long)e << 52));
}

AIRGA_LEAN double rsqrt1(double d) {
    const unsigned long long b = bits_of(d);
    if (b == 0ull) return 0.0;
    const int E = (int)((b >> 52) & 0x7FFu) - 1023;
    const int k = E >> 1;
    const int r = E - 2 * k;
    const double m = from_bits((b & 0x000FFFFFFFFFFFFFull) | ((unsigned long long)(1023 + r) << 52));
    const unsigned yb = f_bits(rsqrt_seed(reduced_to_f32(bits_of(m))));
    double y = from_bits(((unsigned long long)(((yb >> 23) & 0xFFu) - 127u + 1023u) << 52) |
                         ((unsigned long long)(yb & 0x7FFFFFu) << 29));
    const double h = from_bits(bits_of(m) - (1ull << 52));
    y = fma(y, fma(-(h * y), y, 0.5), y);
    return from_bits(bits_of(y) - ((unsigned long long)(long long)k << 52));
}

#if defined(__CUDACC__)
// IEEE division, kept out of line so the compiler never executes it
// speculatively on the fast path of rcp_signed
static __device__ __noinline__ double rcp_ieee(double d) { return 1.0 / d; }
#else
inline double rcp_ieee(double d) { return 1.0 / d; }
#endif

// 1/d for any nonzero finite d: sign by bit operations, the two-step rcp for
// |d| in [2^-1000, 2^1000], the IEEE division otherwise (rare)
AIRGA_LEAN double rcp_signed(double d) {
    const unsigned long long b = bits_of(d);
    const unsigned ex = (unsigned)(b >> 52) & 0x7FFu;
    if (ex < 23u || ex > 2023u) return rcp_ieee(d);
    const double r = rcp(from_bits(b & 0x7FFFFFFFFFFFFFFFull));
    return from_bits(bits_of(r) | (b & 0x8000000000000000ull));
}

// x with the sign of -s (s's sign bit inverted), |x| assumed: for x >= 0
AIRGA_LEAN double neg_sign_of(double x, double s) {
    return from_bits(bits_of(x) | (~bits_of(s) & 0x8000000000000000ull));
}

AIRGA_LEAN double abs_of(double x) { return from_bits(bits_of(x) & 0x7FFFFFFFFFFFFFFFull); }

}  // namespace lean
}  // namespace airga
