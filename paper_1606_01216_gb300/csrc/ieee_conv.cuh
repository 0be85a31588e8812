// IEEE-754 binary64 <-> binary32 conversions and exact halving written with
// integer operations only, usable in device code and (for testing) in host
// C++.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define AIRGA_HD __device__ __forceinline__
#else
#include <cstring>
#define AIRGA_HD inline
namespace airga {
namespace ieee {
namespace hostshim {
inline long long dbl_as_ll(double d) { long long u; std::memcpy(&u, &d, 8); return u; }
inline double ll_as_dbl(long long u) { double d; std::memcpy(&d, &u, 8); return d; }
inline float uint_as_flt(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
inline unsigned flt_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
inline double hilo(int h, int l) { return ll_as_dbl((long long)(((unsigned long long)(unsigned)h << 32) | (unsigned)l)); }
inline int clz32(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
}  // namespace hostshim
}  // namespace ieee
}  // namespace airga
#define __double_as_longlong(x) airga::ieee::hostshim::dbl_as_ll(x)
#define __longlong_as_double(x) airga::ieee::hostshim::ll_as_dbl(x)
#define __uint_as_float(x) airga::ieee::hostshim::uint_as_flt(x)
#define __float_as_uint(x) airga::ieee::hostshim::flt_as_uint(x)
#define __hiloint2double(h, l) airga::ieee::hostshim::hilo(h, l)
#define __clz(x) airga::ieee::hostshim::clz32(x)
#endif

namespace airga {
namespace ieee {

// IEEE-754 conversions between binary64 and binary32, and exact halving,
// written with integer operations only.  On this GPU the FP64 pipe executes 2
// operations per clock per SM and also carries the conversion instructions,
// which made them the bottleneck of the learned build (the compiler executes
// both sides of a rarely taken branch, so even a fallback conversion costs
// its full price); the integer pipes are many times wider.
//   f64_to_f32: round to nearest, ties to even, for every input (overflow
//               gives +-inf, NaN stays NaN, subnormal results are rounded).
//   f32_to_f64: exact for every input (zeros, subnormals, inf, NaN included).
//   half_of:    x / 2 exactly as IEEE division rounds it (ties to even).
AIRGA_HD float f64_to_f32(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const unsigned ex = (hi >> 20) & 0x7FFu;
    const int e = (int)ex - 1023 + 127;
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 of the 52 fraction bits
    const unsigned rem = lo & 0x1FFFFFFFu;                     // the 29 dropped bits
    unsigned r;
    if (ex == 0x7FFu) r = sign | 0x7F800000u | ((((hi & 0xFFFFFu) | lo) != 0u) ? 0x00400000u | m : 0u);
    else if (e >= 255) r = sign | 0x7F800000u;
    else if (e <= 0) {                        // binary32 subnormal (or zero) result
        const int sh = 30 - e;                    // drop 29 + (1 - e) bits of the 53-bit significand
        if (sh > 54) {
            r = sign;
        } else {
            const unsigned long long M = (1ull << 52) | (b & 0x000FFFFFFFFFFFFFull);
            const unsigned long long q = M >> sh, rm = M & ((1ull << sh) - 1ull), hv = 1ull << (sh - 1);
            r = sign | (unsigned)(q + ((rm > hv || (rm == hv && (q & 1ull))) ? 1ull : 0ull));
        }
    } else {
        r = sign | ((unsigned)e << 23) | m;
        r += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;   // may carry into the exponent
    }
    return __uint_as_float(r);
}

AIRGA_HD double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned hi, lo;
    if (e == 0u && m == 0u) {
        hi = sign;
        lo = 0u;
    } else if (e == 0xFFu) {
        hi = sign | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else {
        int e64 = (int)e - 127 + 1023;
        if (e == 0u) {                               // subnormal: normalise
            const int sh = __clz((int)m) - 8;        // bring the leading 1 to bit 23
            m = (m << sh) & 0x7FFFFFu;
            e64 = 1 - 127 + 1023 - sh;
        }
        hi = sign | ((unsigned)e64 << 20) | (m >> 3);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

AIRGA_HD double half_of(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sign = b & 0x8000000000000000ull;
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    if (e == 0x7FFu) return x;                                   // inf, NaN
    if (e > 1u) return __longlong_as_double((long long)(b - (1ull << 52)));
    // zero, subnormal or the smallest normal binade: shift the significand
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (e == 1u ? (1ull << 52) : 0ull);
    const unsigned long long h = (m >> 1) + ((m & 1ull) & ((m >> 1) & 1ull));
    return __longlong_as_double((long long)(sign | h));
}

}  // namespace ieee
}  // namespace airga
