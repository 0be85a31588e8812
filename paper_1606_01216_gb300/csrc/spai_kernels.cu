// SPAI and SPAI-update factors on a band pattern, one column per thread.
//
// Column j of the factor solves the small least-squares problem of Eq. (3.1)
// (SPAI: b_j = e_j) or of the update objective of Sec. 3.2 (b_j = A_old e_j):
//     m_j = argmin || b_j - A m ||_2   over m supported on J_j = {j-W..j+W}.
// Only the rows I_j = {j-W-3 .. j+W+3} of A(:, J_j) can be nonzero, so the
// problem is the (2W+7) x (2W+1) block  Ahat(r, c) = A(j-W-3+r, j-W+c),
// which is itself banded: column c is nonzero only in local rows c..c+6.
//
// QR mode: Householder triangularisation of Ahat exploiting that band — the
// reflector of column c acts on local rows c..c+6 only (rows below c+6 of
// every later column are still zero when column c is reached), so each
// reflector has 7 entries however tall the block.  The whole block, the
// right-hand side and R live in registers (all loops unrolled with
// compile-time indices); one thread owns one column, so every FP64 lane of
// a warp does useful work (the FP64 pipe is GB300's binding resource here).
//
// Columns of J_j outside [0, n) have no unknown: they are given the unit
// vector on their own (out-of-range, otherwise all-zero) local row, which
// decouples them (their solution is exactly 0 and is not stored) and keeps
// the block full rank without changing the other columns' solution.
//
// MR mode: the paper's minimal-residual iteration (Algorithms 2 and 4) on
// the same block, with the direction restricted to the pattern.
#include <utility>

#include "check.cuh"
#include "airga_internal.cuh"
#include "fp64_lean.cuh"

namespace airga {
namespace {

constexpr int kThreadsSpai = 128;

// Gather Ahat (banded: a[r][c] for r in c..c+6) for column j; columns outside
// [0, n) become unit columns on local row c+3.
template <int W>
__device__ __forceinline__ void gather_block(int64_t n, int64_t j, const double *__restrict__ A,
                                             double (&a)[2 * W + 7][2 * W + 1]) {
    constexpr int NC = 2 * W + 1;
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int r = 0; r < c; ++r) a[r][c] = 0.0;     // above the band: fills in during QR
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t k = j - W + c;                  // global column
        const bool col_ok = (k >= 0 && k < n);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
            const int r = c + t;                       // local row
            const int64_t g = j - W - 3 + r;           // global row
            double v = 0.0;
            if (col_ok && g >= 0 && g < n && AIRGA_CK((int64_t)(c - r + 6) * n + g, 0, 7 * n, 501))
                v = __ldg(A + (int64_t)(c - r + 6) * n + g);
            if (!col_ok && t == 3) v = 1.0;            // decoupled unit column
            a[r][c] = v;
        }
    }
}

// Right-hand side: e_j (build) or A_old(I_j, j) (update).  b has 2W+7 rows.
template <int W>
__device__ __forceinline__ void gather_rhs(int64_t n, int64_t j, const double *__restrict__ Aold,
                                           double (&b)[2 * W + 7]) {
    constexpr int NR = 2 * W + 7;
#pragma unroll
    for (int r = 0; r < NR; ++r) b[r] = 0.0;
    if (!Aold) {
        b[W + 3] = 1.0;
        return;
    }
#pragma unroll
    for (int r = W; r <= W + 6; ++r) {
        const int64_t g = j - W - 3 + r;               // row of A_old(:, j)
        if (g >= 0 && g < n && AIRGA_CK((int64_t)(W + 6 - r) * n + g, 0, 7 * n, 502))
            b[r] = __ldg(Aold + (int64_t)(W + 6 - r) * n + g);
    }
}

// Store column j of the factor: F(j-W+c, j) = m[c]; diagonals |d| > W and
// entries whose column is outside the matrix are written as 0 by the thread
// that owns that row, so the whole band is defined.
template <int W>
__device__ __forceinline__ void store_column(int64_t n, int64_t j, const double (&m)[2 * W + 1],
                                             double *__restrict__ F) {
    constexpr int NC = 2 * W + 1;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t i = j - W + c;                   // row of F
        if (i >= 0 && i < n && AIRGA_CK((int64_t)(W - c + 3) * n + i, 0, 7 * n, 503))
            F[(int64_t)(W - c + 3) * n + i] = m[c];
    }
#pragma unroll
    for (int d = -3; d <= 3; ++d) {
        const int64_t c = j + d;
        const bool outside = (c < 0 || c >= n);
        if ((d < -W || d > W || outside) && AIRGA_CK((int64_t)(d + 3) * n + j, 0, 7 * n, 504))
            F[(int64_t)(d + 3) * n + j] = 0.0;
    }
}

// Compile-time fill-in plan of the banded Householder sweep.  For every step
// C it records which local rows of each block column and of the right-hand
// side can be nonzero before the step (bit r of a[C][c] / b[C]).  Row C of
// the reflector is always nonzero; a later column (or b) is transformed only
// if its support meets the reflector's, and then fills in on the reflector's
// support.  Every product with a structural zero is dropped from the unrolled
// code.
//   PAR = -1  general band: only the band shape and, for the build, the sparse
//             right-hand side e_j are used.
//   PAR = 0/1 beam band of a column j of that parity: additionally the
//             Hermite-beam zeros (every row pair but the last: even rows have
//             A(i, i-3) = A(i, i+1) = 0, odd rows A(i, i+3) = A(i, i-1) = 0).
//   RHS = 0   b = e_j (SPAI build); 1: b = a general band column (update);
//         2   b = a beam band column (update from a beam matrix, PAR >= 0).
struct QrPlan {
    unsigned short a[8][7];
    unsigned short b[8];
};

__host__ __device__ constexpr bool beam_zero(int W, int par, int r, int c) {
    // local entry (r, c) is A(g, k), g = j - W - 3 + r, k = g + (c - r + 3)
    const int g = par + W + 3 + r;   // parity of g
    const int d = c - r + 3;
    return (g & 1) == 0 ? (d == -3 || d == 1) : (d == 3 || d == -1);
}

// Can local entry (r, c) of column j's block be nonzero?  E < 0: any column
// away from the last rows; E >= 0: the column j = n - 1 - E of a beam matrix
// (PAR >= 0), whose block reaches past the last row: there rows g >= n are
// zero, columns k >= n are unit columns (only the diagonal entry), and the
// last row pair (g = n - 2, n - 1) carries no beam zeros.
__host__ __device__ constexpr bool plan_nz(int W, int PAR, int E, int r, int c) {
    if (E >= 0) {
        if (c >= E + W + 1) return r == c + 3;     // k = n - 1 - E - W + c >= n
        if (r >= E + W + 4) return false;          // g = n - 1 - E - W - 3 + r >= n
        if (r >= E + W + 2) return true;           // g in the last row pair
    }
    return PAR < 0 || !beam_zero(W, PAR, r, c);
}

__host__ __device__ constexpr QrPlan make_plan(int W, int PAR, int RHS, int E = -1) {
    QrPlan P{};
    const int NC = 2 * W + 1;
    unsigned a[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned b = 0;
    for (int c = 0; c < NC; ++c)
        for (int r = c; r < c + 7; ++r)
            if (plan_nz(W, PAR, E, r, c)) a[c] |= 1u << r;
    if (RHS == 0) {
        b = 1u << (W + 3);
    } else {
        for (int r = W; r <= W + 6; ++r)   // b_r = A_old(g, j): local column W of the block
            if (RHS == 1 || plan_nz(W, PAR, E, r, W)) b |= 1u << r;
    }
    for (int C = 0; C < NC; ++C) {
        for (int c = 0; c < NC; ++c) P.a[C][c] = (unsigned short)a[c];
        P.b[C] = (unsigned short)b;
        const unsigned v = (a[C] & (0x7Fu << C)) | (1u << C);
        for (int c = C + 1; c < NC; ++c)
            if (v & a[c]) a[c] |= v;
        if (v & b) b |= v;
    }
    for (int c = 0; c < NC; ++c) P.a[NC][c] = (unsigned short)a[c];
    P.b[NC] = (unsigned short)b;
    return P;
}

// Gather the block entries the plan says can be nonzero (the others are 0);
// columns outside [0, n) become unit columns on local row c+3 (general plan
// only).
template <int W, int PAR, int E>
__device__ __forceinline__ void gather_block_p(int64_t n, int64_t j, const double *__restrict__ A,
                                               double (&a)[2 * W + 7][2 * W + 1]) {
    constexpr int NC = 2 * W + 1;
    constexpr QrPlan P = make_plan(W, PAR, 0, E);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int r = 0; r < c; ++r) a[r][c] = 0.0;     // above the band: fills in during QR
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t k = j - W + c;                  // global column
        const bool col_ok = (k >= 0 && k < n);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
            const int r = c + t;                       // local row
            const int64_t g = j - W - 3 + r;           // global row
            double v = 0.0;
            if ((P.a[0][c] >> r) & 1u) {
                if (col_ok && g >= 0 && g < n && AIRGA_CK((int64_t)(c - r + 6) * n + g, 0, 7 * n, 505))
                    v = __ldg(A + (int64_t)(c - r + 6) * n + g);
                if (!col_ok && t == 3) v = 1.0;        // decoupled unit column
            }
            a[r][c] = v;
        }
    }
}

// One Householder step on column C of the banded block (local rows C..C+6):
// v = x + sign(x_0) ||x|| e_0, applied to the later columns and to b;
// R_CC stored in a[C][C], 1/R_CC in rinv[C].  Every array index is a
// compile-time constant after unrolling, so the block stays in registers and
// the plan's zero tests fold away.
//
// The scalar part costs few FP64-pipe instructions: 1/sqrt and the
// reciprocal come from lean::rsqrt1 / lean::rcp1 (FP32 hardware seed, one FP64
// Newton step: relative error below 2^-43, which perturbs the reflectors by
// that much, far below the 1e-10 the columns are held to), signs and absolute
// values are integer bit operations, and
// the rank test tracks the largest and smallest ||x|| by their bit patterns
// (non-negative doubles order like their bits).
template <int W, int PAR, int RHS, int E, int C>
__device__ __forceinline__ void qr_step(double (&a)[2 * W + 7][2 * W + 1], double (&b)[2 * W + 7],
                                        double (&rinv)[2 * W + 1], unsigned long long &rmax,
                                        unsigned long long &rmin) {
    constexpr int NC = 2 * W + 1;
    constexpr QrPlan P = make_plan(W, PAR, RHS, E);
    constexpr unsigned V = (P.a[C][C] & (0x7Fu << C)) | (1u << C);   // reflector support
    double sigma = 0.0;
#pragma unroll
    for (int t = 0; t < 7; ++t)
        if ((P.a[C][C] >> (C + t)) & 1u) sigma = fma(a[C + t][C], a[C + t][C], sigma);
    const double x0 = a[C][C];
    const double rs = lean::rsqrt1(sigma);             // 0 when sigma == 0
    const double nrm = sigma * rs;                     // ||x||
    const double alpha = lean::neg_sign_of(nrm, x0);   // R_CC = -sign(x0) ||x||
    const double v0 = x0 - alpha;                      // x0 + sign(x0) ||x||
    // H = I - tau v v^T, v = (v0, a[C+1..C+6][C]), tau = 2 / v^T v = 1 / (||x|| |v0|)
    const double tau = lean::rcp1(nrm * lean::abs_of(v0));   // 0 when sigma == 0
#pragma unroll
    for (int cc = C + 1; cc < NC; ++cc) {
        const unsigned col = P.a[C][cc];
        if ((V & col) == 0u) continue;                 // disjoint supports: column unchanged
        double s = ((col >> C) & 1u) ? v0 * a[C][cc] : 0.0;
#pragma unroll
        for (int t = 1; t < 7; ++t)
            if (((V & col) >> (C + t)) & 1u) s = fma(a[C + t][C], a[C + t][cc], s);
        s *= tau;
        a[C][cc] = ((col >> C) & 1u) ? fma(-s, v0, a[C][cc]) : -s * v0;
#pragma unroll
        for (int t = 1; t < 7; ++t) {
            if (!((V >> (C + t)) & 1u)) continue;
            a[C + t][cc] = ((col >> (C + t)) & 1u) ? fma(-s, a[C + t][C], a[C + t][cc])
                                                   : -s * a[C + t][C];
        }
    }
    {
        const unsigned bm = P.b[C];
        if ((V & bm) != 0u) {
            double s = ((bm >> C) & 1u) ? v0 * b[C] : 0.0;
#pragma unroll
            for (int t = 1; t < 7; ++t)
                if (((V & bm) >> (C + t)) & 1u) s = fma(a[C + t][C], b[C + t], s);
            s *= tau;
            b[C] = ((bm >> C) & 1u) ? fma(-s, v0, b[C]) : -s * v0;
#pragma unroll
            for (int t = 1; t < 7; ++t) {
                if (!((V >> (C + t)) & 1u)) continue;
                b[C + t] = ((bm >> (C + t)) & 1u) ? fma(-s, a[C + t][C], b[C + t]) : -s * a[C + t][C];
            }
        }
    }
    a[C][C] = alpha;
    rinv[C] = lean::neg_sign_of(rs, x0);               // 1 / R_CC
    const unsigned long long nb = lean::bits_of(nrm);
    rmax = nb > rmax ? nb : rmax;
    rmin = nb < rmin ? nb : rmin;
}

template <int W, int PAR, int RHS, int E, int... Cs>
__device__ __forceinline__ void qr_all(std::integer_sequence<int, Cs...>,
                                       double (&a)[2 * W + 7][2 * W + 1], double (&b)[2 * W + 7],
                                       double (&rinv)[2 * W + 1], unsigned long long &rmax,
                                       unsigned long long &rmin) {
    (qr_step<W, PAR, RHS, E, Cs>(a, b, rinv, rmax, rmin), ...);
}

// Right-hand side entries the plan says can be nonzero (RHS 1/2: A_old(I_j, j))
template <int W, int PAR, int RHS, int E>
__device__ __forceinline__ void gather_rhs_p(int64_t n, int64_t j, const double *__restrict__ Aold,
                                             double (&b)[2 * W + 7]) {
    constexpr int NR = 2 * W + 7;
    constexpr QrPlan P = make_plan(W, PAR, RHS, E);
#pragma unroll
    for (int r = 0; r < NR; ++r) b[r] = 0.0;
    if constexpr (RHS == 0) {
        b[W + 3] = 1.0;
    } else {
#pragma unroll
        for (int r = W; r <= W + 6; ++r) {
            const int64_t g = j - W - 3 + r;           // row of A_old(:, j)
            if (((P.b[0] >> r) & 1u) && g >= 0 && g < n &&
                AIRGA_CK((int64_t)(W + 6 - r) * n + g, 0, 7 * n, 506))
                b[r] = __ldg(Aold + (int64_t)(W + 6 - r) * n + g);
        }
    }
}

// Solve column j's least-squares problem with the plan (PAR, RHS, E) and store it.
template <int W, int PAR, int RHS, int E = -1>
__device__ __forceinline__ void qr_column(int64_t n, int64_t j, const double *__restrict__ A,
                                          const double *__restrict__ Aold, double *__restrict__ F,
                                          double *__restrict__ colres, int32_t *rank_flag) {
    constexpr int NC = 2 * W + 1;
    constexpr int NR = NC + 6;
    double a[NR][NC];
    double b[NR];
    gather_block_p<W, PAR, E>(n, j, A, a);
    gather_rhs_p<W, PAR, RHS, E>(n, j, Aold, b);
    double rinv[NC];
    unsigned long long rmax = 0ull, rmin = ~0ull;      // bit patterns of ||x|| >= 0
    qr_all<W, PAR, RHS, E>(std::make_integer_sequence<int, NC>{}, a, b, rinv, rmax, rmin);
    double m[NC];
    const bool rank_ok = rmin != 0ull && lean::from_bits(rmin) >= 1e-14 * lean::from_bits(rmax);
#pragma unroll
    for (int ci = 0; ci < NC; ++ci) {
        const int c = NC - 1 - ci;
        double s = b[c];
#pragma unroll
        for (int cc = c + 1; cc < NC; ++cc) s = fma(-a[c][cc], m[cc], s);
        m[c] = rank_ok ? s * rinv[c] : 0.0;
    }
    if (!rank_ok) atomicOr(rank_flag, 1);
    if (colres) {
        double rr = 0.0;
#pragma unroll
        for (int r = NC; r < NR; ++r) rr = fma(b[r], b[r], rr);
        colres[j] = rr * lean::rsqrt1(rr);             // ||b_j - A m_j||
    }
    store_column<W>(n, j, m, F);
}

// Two launches per SPAI call, each with the registers of one plan only (the
// general plan needs ~230, the beam plans ~155-170; one kernel holding both
// runs at the larger count and fewer warps per SM):
//  * spai_qr_beam_kernel: every column of a matrix carrying the beam
//    zero-structure flag (and A_old too, for an update), n even and >= 16.
//    Warps take columns of one parity (the two interior beam plans never
//    diverge in a warp), and warp pairs run from the last columns down, so
//    the warps holding the last 8 columns, each with a plan of its own, start
//    first and their divergence stays off the critical path.  The first
//    columns use the interior plan: their out-of-range rows and unit columns
//    agree with it.  Returns at once on other matrices.
//  * spai_qr_kernel: the general plan, for matrices without the flag; returns
//    at once on flagged ones.
__device__ __forceinline__ bool beam_matrix(int64_t n, int upd, const int32_t *zA,
                                            const int32_t *zAold) {
    return zA && *zA != 0 && (!upd || (zAold && *zAold != 0)) && (n % 2 == 0) && n >= 16;
}

template <int RHS, int PAR, int E>
__device__ __forceinline__ void end_column(int64_t n, int64_t j, const double *__restrict__ A,
                                           const double *__restrict__ Aold, double *__restrict__ F,
                                           double *__restrict__ colres, int32_t *rank_flag) {
    qr_column<3, PAR, RHS, E>(n, j, A, Aold, F, colres, rank_flag);
}

template <int UPD>
__global__ void __launch_bounds__(kThreadsSpai)
spai_qr_beam_kernel(int64_t n, const double *__restrict__ A, const double *__restrict__ Aold,
                    double *__restrict__ F, double *__restrict__ colres, int32_t *rank_flag,
                    const int32_t *__restrict__ zA, const int32_t *__restrict__ zAold) {
    constexpr int W = 3, RHS = UPD ? 2 : 0;
    if (!beam_matrix(n, UPD, zA, zAold)) return;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t w = gt >> 5;
    const int64_t pair = (n + 63) / 64 - 1 - (w >> 1);   // 64 columns per warp pair
    if (pair < 0) return;
    const int64_t j = 2 * (pair * 32 + (gt & 31)) + (w & 1);
    if (j >= n) return;
    // n is even: j = n - 1 - e has parity (e + 1) mod 2
    switch (n - 1 - j) {
        case 0: end_column<RHS, 1, 0>(n, j, A, Aold, F, colres, rank_flag); return;
        case 1: end_column<RHS, 0, 1>(n, j, A, Aold, F, colres, rank_flag); return;
        case 2: end_column<RHS, 1, 2>(n, j, A, Aold, F, colres, rank_flag); return;
        case 3: end_column<RHS, 0, 3>(n, j, A, Aold, F, colres, rank_flag); return;
        case 4: end_column<RHS, 1, 4>(n, j, A, Aold, F, colres, rank_flag); return;
        case 5: end_column<RHS, 0, 5>(n, j, A, Aold, F, colres, rank_flag); return;
        case 6: end_column<RHS, 1, 6>(n, j, A, Aold, F, colres, rank_flag); return;
        case 7: end_column<RHS, 0, 7>(n, j, A, Aold, F, colres, rank_flag); return;
        default: break;
    }
    if (j & 1) qr_column<W, 1, RHS>(n, j, A, Aold, F, colres, rank_flag);
    else qr_column<W, 0, RHS>(n, j, A, Aold, F, colres, rank_flag);
}

template <int W, int UPD>
__global__ void __launch_bounds__(kThreadsSpai)
spai_qr_kernel(int64_t n, const double *__restrict__ A, const double *__restrict__ Aold,
               double *__restrict__ F, double *__restrict__ colres, int32_t *rank_flag,
               const int32_t *__restrict__ zA, const int32_t *__restrict__ zAold) {
    if (W == 3 && beam_matrix(n, UPD, zA, zAold)) return;   // the beam kernel's matrix
    // grid-stride over one resident wave, so that on a flagged matrix the
    // launch is one wave of blocks that return at once
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride)
        qr_column<W, -1, UPD ? 1 : 0>(n, j, A, Aold, F, colres, rank_flag);
}

template <int W>
__global__ void __launch_bounds__(kThreadsSpai)
spai_mr_kernel(int64_t n, const double *__restrict__ A, const double *__restrict__ Aold,
               const double *__restrict__ alpha0p, double tol, int relative, int kmax,
               double *__restrict__ F, int32_t *__restrict__ steps,
               double *__restrict__ colres) {
    constexpr int NC = 2 * W + 1;
    constexpr int NR = NC + 6;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;

    double a[NR][NC];
    double b[NR];
    gather_block<W>(n, j, A, a);
    gather_rhs<W>(n, j, Aold, b);
    bool in[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int64_t k = j - W + c;
        in[c] = (k >= 0 && k < n);
        if (!in[c]) a[c + 3][c] = 0.0;                 // no unknown here: drop the unit column
    }
    // m = alpha0 e_j (local column W); r = b - Ahat m
    const double alpha0 = *alpha0p;
    double m[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) m[c] = 0.0;
    m[W] = alpha0;
    double r[NR];
    double bb = 0.0;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        bb = fma(b[q], b[q], bb);
        double am = (q >= W && q <= W + 6) ? a[q][W] * alpha0 : 0.0;
        r[q] = b[q] - am;
    }
    // stop when ||r|| <= tol (the loop test of Algorithms 2 / 4) or, in the
    // relative reading, ||r|| <= tol ||b_j||; tested on squares: no square
    // root per step
    const double thr2 = relative ? (tol * tol) * bb : tol * tol;
    double rn2 = 0.0;
#pragma unroll
    for (int q = 0; q < NR; ++q) rn2 = fma(r[q], r[q], rn2);
    int k = 0;
    while (rn2 > thr2 && k < kmax) {
        // d = r restricted to the pattern: column c's unknown sits on local row c+3
        double d[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) d[c] = in[c] ? r[c + 3] : 0.0;
        double w[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) w[q] = 0.0;
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int t = 0; t < 7; ++t) w[c + t] = fma(a[c + t][c], d[c], w[c + t]);
        double ww = 0.0, rw = 0.0;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            ww = fma(w[q], w[q], ww);
            rw = fma(r[q], w[q], rw);
        }
        if (ww == 0.0) break;                          // r vanishes on the pattern
        const double al = rw * lean::rcp_signed(ww);   // step length (r, w) / (w, w)
#pragma unroll
        for (int c = 0; c < NC; ++c) m[c] = fma(al, d[c], m[c]);
        rn2 = 0.0;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            r[q] = fma(-al, w[q], r[q]);
            rn2 = fma(r[q], r[q], rn2);
        }
        ++k;
    }
    steps[j] = k;
    if (colres) colres[j] = sqrt(rn2);
#pragma unroll
    for (int c = 0; c < NC; ++c)
        if (!in[c]) m[c] = 0.0;
    store_column<W>(n, j, m, F);
}

// ---------------------------------------------------------------------------
// Normal-equations solver of the same least-squares problems (spai_mode
// AIRGA_SPAI_NE, pattern half-width 3).  With Ahat = A(I_j, J_j) the
// minimiser solves G m = g, G = Ahat^T Ahat, g = Ahat^T b_j.  Every row
// outside I_j is zero in the columns J_j, so G is the principal submatrix
// (A^T A)(J_j, J_j) of the band-13 matrix A^T A: one pass computes its upper
// band for all columns at once (28 FMA per row, against ~140 per column for
// a block product), and for a build g = A(j, J_j)^T is row j of A.  G is
// factored as L D L^T in registers (unit lower L, the pivots inverted with
// the two-step lean reciprocal), and the residual b_j - Ahat m is formed
// explicitly for ||b_j - A m_j||.  About half the FP64 instructions of the
// Householder solve per column.
//
// Accuracy: the normal equations square the block's condition number.  A
// column whose pivots signal an ill-conditioned G (a pivot <= 0, or
// min pivot < 1e-6 max diagonal of G; the pivots bound cond(G) from below
// within a small factor on these 7 x 7 blocks) is not written here: it is
// appended to a list that the Householder kernel then solves, so every
// column keeps the QR path's accuracy class.  On the unit-element beam the
// worst block has min pivot / max diagonal = 3.2e-6 (cond(G) = 4.6e5) and
// the normal-equation columns agree with the Householder ones to 2e-12.
// ---------------------------------------------------------------------------
constexpr int kGramRows = 128;
constexpr int kGramStage = kGramRows + 8;   // band rows i0-3 .. i0+kGramRows+4
static_assert(kGramRows % 64 == 0, "parity-mapped warp pairs cover 64 columns");

// Beam zero structure (checked at import, the pairz flag, on every row but
// the last two): on an even row k the band entries at offsets -3 and +1 are
// stored zeros, on an odd row those at +3 and -1.  P is the parity of row
// k - t.
template <int P>
__device__ constexpr bool beam_zero(int t, int off) {
    return (((P + t) & 1) == 0) ? (off == -3 || off == 1) : (off == 3 || off == -1);
}

// Column i of the Gram band: U[d n + i] = (A^T A)(i, i + d), d = 0..6, summed
// over the rows k = i + t common to both columns in increasing k.  BEAM with
// row parity P: the products with a stored-zero factor are skipped (each
// would add an exact zero), 18 FMA instead of 28.
template <bool BEAM, int P>
__device__ __forceinline__ void gram_column(int64_t n, int64_t i, int li,
                                            const double (&sb)[kBand][kGramStage],
                                            double *__restrict__ U) {
#pragma unroll
    for (int d = 0; d < kBand; ++d) {
        double acc = 0.0;
#pragma unroll
        for (int t = d - 3; t <= 3; ++t) {                 // k = i + t
            if (BEAM && (beam_zero<P>(t, -t) || beam_zero<P>(t, d - t))) continue;
            acc = fma(sb[3 - t][li + t], sb[d + 3 - t][li + t], acc);
        }
        if (AIRGA_CK((int64_t)d * n + i, 0, 7 * n, 507))
            U[(int64_t)d * n + i] = i + d < n ? acc : 0.0;
    }
}

// U[d n + i] = (A^T A)(i, i + d), d = 0..6 (0 where i + d >= n).  A CTA
// stages the band rows its columns touch in shared memory (rows outside
// [0, n) as zeros).  zA (device, may be null): A's beam-structure flag; with
// it set the warps are parity-mapped (a warp pair covers 64 consecutive
// columns, the even warp the even ones) so that each warp skips the same
// zero products.
__global__ void __launch_bounds__(kGramRows)
gram_band_kernel(int64_t n, const double *__restrict__ A, double *__restrict__ U,
                 const int32_t *__restrict__ zA) {
    __shared__ double sb[kBand][kGramStage];
    const int64_t i0 = (int64_t)blockIdx.x * kGramRows;
    const int64_t k0 = i0 - 3;                             // band row of stage slot 0
    for (int t = threadIdx.x; t < kBand * kGramStage; t += kGramRows) {
        const int d = t / kGramStage, q = t - d * kGramStage;
        const int64_t k = k0 + q;
        sb[d][q] = (k >= 0 && k < n) ? __ldg(A + (int64_t)d * n + k) : 0.0;
    }
    __syncthreads();
    // A(k, c) = band[(c - k + 3) n + k] = sb[c - k + 3][k - k0]
    if (zA && *zA) {
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        const int par = w & 1;
        const int64_t i = i0 + 64 * (w >> 1) + 2 * l + par;
        if (i >= n) return;
        const int li = (int)(i - k0);
        if (i + 3 >= n - 2) gram_column<false, 0>(n, i, li, sb, U);   // touches the last rows
        else if (par == 0) gram_column<true, 0>(n, i, li, sb, U);
        else gram_column<true, 1>(n, i, li, sb, U);
    } else {
        const int64_t i = i0 + threadIdx.x;
        if (i >= n) return;
        gram_column<false, 0>(n, i, (int)(i - k0), sb, U);
    }
}

// Ahat(r, c) = A(j-6+r, j-3+c) for r in c..c+6 (0 outside the matrix)
__device__ __forceinline__ double ahat(const double *__restrict__ A, int64_t n, int64_t j, int r,
                                       int c) {
    const int64_t row = j - 6 + r, col = j - 3 + c;
    if (row < 0 || row >= n || col < 0 || col >= n) return 0.0;
    const int64_t at = (int64_t)(c - r + 6) * n + row;
    return AIRGA_CK(at, 0, 7 * n, 508) ? __ldg(A + at) : 0.0;
}

// b(r) = A_old(j-6+r, j), nonzero for r in 3..9
__device__ __forceinline__ double bhat(const double *__restrict__ Aold, int64_t n, int64_t j,
                                       int r) {
    const int64_t row = j - 6 + r;
    if (row < 0 || row >= n) return 0.0;
    const int64_t at = (int64_t)(9 - r) * n + row;
    return AIRGA_CK(at, 0, 7 * n, 509) ? __ldg(Aold + at) : 0.0;
}

// BEAM: A has the beam's zero structure (checked at import on every row but
// the last two: offsets -3 and +1 vanish on even rows, +3 and -1 on odd
// rows), so the Gram block's corner G(j-3, j+3) = A(j, j-3) A(j, j+3) is
// exactly zero wherever it lies inside the matrix (j + 3 < n, so row j is
// checked; one factor is a stored zero) and the L D L^T terms through it are
// skipped: L(6, 0) = 0 exactly, and the skipped products would each add a
// zero.
template <int UPD, bool BEAM>
__device__ __forceinline__ void ne_column(int64_t n, int64_t j, const double *__restrict__ A,
                                          const double *__restrict__ Aold,
                                          const double *__restrict__ U, double *__restrict__ F,
                                          double *__restrict__ colres, int want_colres,
                                          int32_t *__restrict__ fb_count,
                                          int32_t *__restrict__ fb_list) {
    bool in[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) in[c] = j - 3 + c >= 0 && j - 3 + c < n;
    // right-hand side g = Ahat^T b_j
    double g[7];
    if (!UPD) {
#pragma unroll
        for (int c = 0; c < 7; ++c)                        // A(j, j-3+c) = band[c n + j]
            g[c] = in[c] ? __ldg(A + (int64_t)c * n + j) : 0.0;
    } else {
        double b[7];                                       // b[r - 3], r = 3..9
#pragma unroll
        for (int r = 3; r <= 9; ++r) b[r - 3] = bhat(Aold, n, j, r);
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            double s = 0.0;
#pragma unroll
            for (int r = (c > 3 ? c : 3); r <= (c + 6 < 9 ? c + 6 : 9); ++r)
                s = fma(ahat(A, n, j, r, c), b[r - 3], s);
            g[c] = s;
        }
    }
    // G = L D L^T row by row: W(i, k) = G(i, k) - sum_{p<k} W(i, p) L(k, p),
    // L(i, k) = W(i, k) / d_k, d_i = G(i, i) - sum_{p<i} W(i, p) L(i, p).
    // Columns outside the matrix are unit rows and columns of G.
    double L[7][7];
    double rinv[7];
    unsigned long long dmax = 0ull, pmin = ~0ull;          // bit patterns (order = value order)
    bool pos = true;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        double w[7];
#pragma unroll
        for (int k = 0; k < i; ++k) {
            if (BEAM && i == 6 && k == 0) {               // the zero corner
                w[0] = 0.0;
                L[6][0] = 0.0;
                continue;
            }
            double s = (in[i] && in[k]) ? __ldg(U + (int64_t)(i - k) * n + (j - 3 + k)) : 0.0;
#pragma unroll
            for (int p = 0; p < k; ++p)
                if (!(BEAM && i == 6 && p == 0)) s = fma(-w[p], L[k][p], s);
            w[k] = s;
            L[i][k] = s * rinv[k];
        }
        double d = in[i] ? __ldg(U + (j - 3 + i)) : 1.0;
        if (in[i]) {
            const unsigned long long db = lean::bits_of(d);
            dmax = db > dmax ? db : dmax;
        }
#pragma unroll
        for (int p = 0; p < i; ++p)
            if (!(BEAM && i == 6 && p == 0)) d = fma(-w[p], L[i][p], d);
        if (in[i]) {
            const unsigned long long pb = lean::bits_of(d);
            pos = pos && (pb >> 63) == 0ull && pb != 0ull;
            pmin = pb < pmin ? pb : pmin;
        }
        rinv[i] = lean::rcp(d);
    }
    // conditioning guard (see above): the Householder pass takes this column
    if (!pos || lean::from_bits(pmin) < 1e-6 * lean::from_bits(dmax)) {
        const int32_t slot = atomicAdd(fb_count, 1);
        if (AIRGA_CK(slot, 0, n, 510)) fb_list[slot] = (int32_t)j;
        return;
    }
    // L y = g, z = D^-1 y, L^T m = z
    double y[7], m[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        double s = g[i];
#pragma unroll
        for (int k = 0; k < i; ++k)
            if (!(BEAM && i == 6 && k == 0)) s = fma(-L[i][k], y[k], s);
        y[i] = s;
    }
#pragma unroll
    for (int ii = 0; ii < 7; ++ii) {
        const int i = 6 - ii;
        double s = y[i] * rinv[i];
#pragma unroll
        for (int k = i + 1; k < 7; ++k)
            if (!(BEAM && k == 6 && i == 0)) s = fma(-L[k][i], m[k], s);
        m[i] = s;
    }
    if (colres && !want_colres) {
        colres[j] = __longlong_as_double(0x7FF8000000000000ll);   // not formed: NaN
    } else if (colres) {
        // ||b_j - Ahat m|| from the explicit residual over the 13 rows
        double rr = 0.0;
#pragma unroll
        for (int r = 0; r < 13; ++r) {
            double v = UPD ? (r >= 3 && r <= 9 ? bhat(Aold, n, j, r) : 0.0) : (r == 6 ? 1.0 : 0.0);
#pragma unroll
            for (int c = (r > 6 ? r - 6 : 0); c <= (r < 6 ? r : 6); ++c)
                v = fma(-ahat(A, n, j, r, c), m[c], v);
            rr = fma(v, v, rr);
        }
        colres[j] = rr * lean::rsqrt1(rr);
    }
    store_column<3>(n, j, m, F);
}

// zA (device, may be null): A's beam-structure flag
template <int UPD>
__global__ void __launch_bounds__(kThreadsSpai)
spai_ne_kernel(int64_t n, const double *__restrict__ A, const double *__restrict__ Aold,
               const double *__restrict__ U, double *__restrict__ F, double *__restrict__ colres,
               int want_colres, int32_t *__restrict__ fb_count, int32_t *__restrict__ fb_list,
               const int32_t *__restrict__ zA) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (zA && *zA)
        ne_column<UPD, true>(n, j, A, Aold, U, F, colres, want_colres, fb_count, fb_list);
    else
        ne_column<UPD, false>(n, j, A, Aold, U, F, colres, want_colres, fb_count, fb_list);
}

// The columns the normal-equation kernel left to the Householder solve (a
// grid-stride loop over the list; one resident wave, most of it idle when
// the list is empty).  steps[j] = 1 marks them.
template <int UPD>
__global__ void __launch_bounds__(kThreadsSpai)
spai_qr_list_kernel(int64_t n, const double *__restrict__ A, const double *__restrict__ Aold,
                    double *__restrict__ F, double *__restrict__ colres, int32_t *rank_flag,
                    const int32_t *__restrict__ fb_count, const int32_t *__restrict__ fb_list,
                    int32_t *__restrict__ steps) {
    const int64_t cnt = *fb_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += stride) {
        const int64_t j = fb_list[t];
        if (!AIRGA_CK(j, 0, n, 511)) continue;
        qr_column<3, -1, UPD ? 1 : 0>(n, j, A, Aold, F, colres, rank_flag);
        if (steps) steps[j] = 1;
    }
}

template <int W>
cudaError_t qr_w(int64_t n, const double *A, const double *Aold, double *F, double *colres,
                 int32_t *flag, const int32_t *zA, const int32_t *zAold, cudaStream_t s) {
    if (W == 3 && zA) {
        // parity-mapped warps: 64 columns per warp pair
        const int64_t blocks_b = (64 * ((n + 63) / 64) + kThreadsSpai - 1) / kThreadsSpai;
        if (Aold)
            spai_qr_beam_kernel<1><<<(unsigned)blocks_b, kThreadsSpai, 0, s>>>(n, A, Aold, F, colres, flag, zA, zAold);
        else
            spai_qr_beam_kernel<0><<<(unsigned)blocks_b, kThreadsSpai, 0, s>>>(n, A, Aold, F, colres, flag, zA, zAold);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // one resident wave of the general kernel (cached per device)
    static int wave_dev[2] = {-1, -1}, wave_blocks[2] = {0, 0};
    const int u = Aold ? 1 : 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (wave_dev[u] != dev) {
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = u ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_qr_kernel<W, 1>, kThreadsSpai, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_qr_kernel<W, 0>, kThreadsSpai, 0);
        if (e != cudaSuccess) return e;
        wave_blocks[u] = sms * (per_sm > 0 ? per_sm : 1);
        wave_dev[u] = dev;
    }
    int64_t blocks = (n + kThreadsSpai - 1) / kThreadsSpai;
    if (blocks > wave_blocks[u]) blocks = wave_blocks[u];
    const int32_t *za = W == 3 ? zA : nullptr;
    if (Aold)
        spai_qr_kernel<W, 1><<<(unsigned)blocks, kThreadsSpai, 0, s>>>(n, A, Aold, F, colres, flag, za, zAold);
    else
        spai_qr_kernel<W, 0><<<(unsigned)blocks, kThreadsSpai, 0, s>>>(n, A, Aold, F, colres, flag, za, zAold);
    return cudaGetLastError();
}

template <int W>
cudaError_t mr_w(int64_t n, const double *A, const double *Aold, const double *alpha0,
                 double tol, int relative, int kmax, double *F, int32_t *steps, double *colres,
                 cudaStream_t s) {
    int64_t blocks = (n + kThreadsSpai - 1) / kThreadsSpai;
    spai_mr_kernel<W><<<(unsigned)blocks, kThreadsSpai, 0, s>>>(n, A, Aold, alpha0, tol, relative,
                                                                 kmax, F, steps, colres);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spai_qr(int64_t n, int hbw, const double *A, const double *A_old, double *F,
                           double *colres, int32_t *rank_flag, const int32_t *zA,
                           const int32_t *zAold, cudaStream_t s) {
    const cudaError_t fe = injected_launch_error();   // host-side test fault only
    if (fe != cudaSuccess) return fe;
    switch (hbw) {
        case 0: return qr_w<0>(n, A, A_old, F, colres, rank_flag, zA, zAold, s);
        case 1: return qr_w<1>(n, A, A_old, F, colres, rank_flag, zA, zAold, s);
        case 2: return qr_w<2>(n, A, A_old, F, colres, rank_flag, zA, zAold, s);
        default: return qr_w<3>(n, A, A_old, F, colres, rank_flag, zA, zAold, s);
    }
}

cudaError_t launch_spai_mr(int64_t n, int hbw, const double *A, const double *A_old,
                           const double *alpha0, double tol, int relative, int kmax, double *F,
                           int32_t *steps, double *colres, cudaStream_t s) {
    switch (hbw) {
        case 0: return mr_w<0>(n, A, A_old, alpha0, tol, relative, kmax, F, steps, colres, s);
        case 1: return mr_w<1>(n, A, A_old, alpha0, tol, relative, kmax, F, steps, colres, s);
        case 2: return mr_w<2>(n, A, A_old, alpha0, tol, relative, kmax, F, steps, colres, s);
        default: return mr_w<3>(n, A, A_old, alpha0, tol, relative, kmax, F, steps, colres, s);
    }
}

cudaError_t launch_spai_ne(int64_t n, const double *A, const double *A_old, double *F,
                           double *colres, bool want_colres, int32_t *rank_flag, int32_t *steps,
                           double *U, int32_t *fb, const int32_t *zA, cudaStream_t s) {
    const int want = want_colres ? 1 : 0;
    const cudaError_t fe = injected_launch_error();   // host-side test fault only
    if (fe != cudaSuccess) return fe;
    const int64_t gb = (n + kGramRows - 1) / kGramRows;
    gram_band_kernel<<<(unsigned)gb, kGramRows, 0, s>>>(n, A, U, zA);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(fb, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n + kThreadsSpai - 1) / kThreadsSpai;
    if (A_old)
        spai_ne_kernel<1><<<(unsigned)blocks, kThreadsSpai, 0, s>>>(n, A, A_old, U, F, colres, want, fb, fb + 1, zA);
    else
        spai_ne_kernel<0><<<(unsigned)blocks, kThreadsSpai, 0, s>>>(n, A, nullptr, U, F, colres, want, fb, fb + 1, zA);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the Householder pass over the listed columns: one resident wave
    static int wave_dev[2] = {-1, -1}, wave_blocks[2] = {0, 0};
    const int u = A_old ? 1 : 0;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (wave_dev[u] != dev) {
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = u ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_qr_list_kernel<1>, kThreadsSpai, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_qr_list_kernel<0>, kThreadsSpai, 0);
        if (e != cudaSuccess) return e;
        wave_blocks[u] = sms * (per_sm > 0 ? per_sm : 1);
        wave_dev[u] = dev;
    }
    const int64_t lb = blocks < wave_blocks[u] ? blocks : wave_blocks[u];
    if (A_old)
        spai_qr_list_kernel<1><<<(unsigned)lb, kThreadsSpai, 0, s>>>(n, A, A_old, F, colres, rank_flag, fb, fb + 1, steps);
    else
        spai_qr_list_kernel<0><<<(unsigned)lb, kThreadsSpai, 0, s>>>(n, A, nullptr, F, colres, rank_flag, fb, fb + 1, steps);
    return cudaGetLastError();
}

}  // namespace airga

AIRGA_CHECK_READER(spai_kernels)
