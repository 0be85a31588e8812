// Bounds-checked builds.  Compiled with -DAIRGA_CHECKED, every instrumented
// memory access first tests its index against the buffer it reads or writes;
// an index outside is recorded (a count, the first site and index) and the
// access is skipped — a load yields 0 — so a wrong index shows up as a
// counter instead of a fault.  In normal builds AIRGA_CK is the constant true
// and costs nothing.
//
// The record lives in a per-translation-unit device array; each instrumented
// file defines one reader with AIRGA_CHECK_READER(name), and
// airga_debug_checked() adds them up.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifdef AIRGA_CHECKED
namespace airga {
namespace ck {
// [0] violations, [1] first site, [2] first index
static __device__ unsigned long long g_check[3];

static __device__ __noinline__ void record(int site, long long idx) {
    if (atomicAdd(&g_check[0], 1ull) == 0ull) {
        g_check[1] = (unsigned long long)site;
        g_check[2] = (unsigned long long)idx;
    }
}

static __device__ __forceinline__ bool in(long long idx, long long lo, long long hi, int site) {
    if (idx >= lo && idx < hi) return true;
    record(site, idx);
    return false;
}
}  // namespace ck
}  // namespace airga

// true when lo <= idx < hi; otherwise records (site, idx) and gives false
#define AIRGA_CK(idx, lo, hi, site) \
    (::airga::ck::in((long long)(idx), (long long)(lo), (long long)(hi), (site)))

// host reader of this translation unit's record: out[0..2], then cleared
#define AIRGA_CHECK_READER(NAME)                                                       \
    namespace airga {                                                                  \
    int check_read_##NAME(unsigned long long *out) {                                   \
        if (cudaMemcpyFromSymbol(out, ck::g_check, sizeof(ck::g_check)) != cudaSuccess) \
            return 1;                                                                  \
        const unsigned long long zero[3] = {0ull, 0ull, 0ull};                         \
        return cudaMemcpyToSymbol(ck::g_check, zero, sizeof(zero)) == cudaSuccess ? 0 : 1; \
    }                                                                                  \
    }
#else
#define AIRGA_CK(idx, lo, hi, site) (true)
#define AIRGA_CHECK_READER(NAME)
#endif
