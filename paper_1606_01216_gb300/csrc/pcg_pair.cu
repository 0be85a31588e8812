// Persistent PCG, node-pair form (shared-memory state, n even).
//
// Same recurrence, ownership, halo and barrier scheme as pcg_kernel.cu (see
// the comment there); what changes is how a CTA walks its rows:
//
// * Each thread owns row PAIRS (i, i+1), i even — for the beam these are the
//   two DOFs (w, theta) of one node.  Band loads are double2 (both rows of a
//   diagonal in one 16-byte load) and the seven window values a pair needs
//   on each side come from five double2 shared-memory loads.
// * Structure-aware A stencil: for the Hermite-cubic beam the band-7 rows
//   have two exact zeros each — the structural +-3 corner and the w_k/theta_k
//   coupling that cancels between neighbouring elements (even rows: offsets
//   -3 and +1; odd rows: +3 and -1; every row but the free-end pair).  When
//   the matrix carries that flag (checked on the device when the matrix is
//   made) the A stencil issues 5 FP64 FMAs per row instead of 7; FP64 issue
//   is the binding resource on GB300 (2 FMA/clk/SM).
// * Reductions use the shared-memory tree of pcg_common.cuh.
//
// Windows (global rows, all bases even so double2 accesses stay aligned):
//   x  [lo, hi)              own rows
//   r  [lo-8, hi+8)          z on own +-4 needs r on own +-7
//   p  [lo-4, hi+4)          q on own rows (and p itself on own +-4)
//   zq [lo-4, hi+4)          z (then q on own rows)
// Out-of-matrix window slots are zero.  Boundary rows of p (first/last 12)
// go to `pbuf` before barrier 1.  The r halo (4 pairs per side) is updated by
// the last 8 threads from p read straight out of `pbuf` (loads issued first)
// and from A's halo rows cached in shared memory at launch; it depends on no
// own-row update, so it runs during the x/r sweep and a single CTA barrier
// precedes z = M r.  Convergence is tested as r.r <= (tol ||b||)^2, keeping
// square roots off the per-iteration critical path; the residual history is
// stored as r.r and converted once at exit.
#include "check.cuh"
#include "fp64_lean.cuh"
#include "pcg_common.cuh"

namespace airga {
namespace {

using namespace pcgdev;

// threads per CTA: the all-shared-memory kernels (single system and batched)
// run at 384, which leaves up to 168 registers per thread for the
// upper-diagonal P_sym read; the split-state kernel, whose windows partly
// live in L2, keeps 512 warps' worth of latency hiding
constexpr int kThreadsFull = 384, kThreadsSplit = 512, kThreadsBatch = 384;
// half-SM split-state kernel (SPLIT == 2): 256 threads and at most half an
// SM's registers and shared memory, so that two solves on different streams
// share every SM and each fills the other's barrier and scalar-chain gaps
constexpr int kThreadsHalf = 256;
constexpr int kThreadsMax = 512;   // sizes the shared-memory reduction buffer
constexpr int HR = 8, HP = 12, HZ = 4;
constexpr int kHaloPairs = HR;   // 4 pairs of r halo on each side

__device__ __forceinline__ void load_band_pair(const double *__restrict__ band, int n,
                                               int i, double2 (&a)[kBand]) {
    if (!AIRGA_CK(i, 0, n - 1, 101)) {          // rows (i, i+1) inside the band arrays
#pragma unroll
        for (int d = 0; d < kBand; ++d) a[d] = make_double2(0.0, 0.0);
        return;
    }
#pragma unroll
    for (int d = 0; d < kBand; ++d)
        a[d] = __ldg(reinterpret_cast<const double2 *>(band + (long long)d * n + i));
}

// v[k] = window row i-4+k, k = 0..9 (five aligned double2 loads); wlen is
// the window's length (checked builds test the ten rows against it)
__device__ __forceinline__ void load_win(const double *w, int wbase, int i,
                                         double (&v)[10], int wlen) {
    if (!AIRGA_CK(i - 4 - wbase, 0, wlen - 9, 102)) {
#pragma unroll
        for (int k = 0; k < 10; ++k) v[k] = 0.0;
        return;
    }
    const double2 *w2 = reinterpret_cast<const double2 *>(w + (i - 4 - wbase));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double2 t = w2[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}

// (y_i, y_{i+1}) = band-7 rows i, i+1 applied to the window values v.
__device__ __forceinline__ double2 pair_full(const double2 (&a)[kBand], const double (&v)[10]) {
    double y0 = a[0].x * v[1], y1 = a[0].y * v[2];
#pragma unroll
    for (int d = 1; d < kBand; ++d) {
        y0 = fma(a[d].x, v[1 + d], y0);
        y1 = fma(a[d].y, v[2 + d], y1);
    }
    return make_double2(y0, y1);
}

// Symmetric band from its upper diagonals U[d][i] = P(i, i+d), d = 0..3 (the
// rows 3n..7n of a band array): the lower entries of pair (i, i+1) are read
// from earlier rows, P(i, i-d) = U[d][i-d], so the band's lower three
// diagonals are never touched and the per-iteration L2 footprint of P_sym
// drops from 56 to 32 B per row.  Products are summed in pair_full's order
// (offsets -3 .. 3), so for a symmetric band the result is the same bit for
// bit.  Out-of-matrix entries multiply window zeros and are not loaded.
__device__ __forceinline__ double2 pair_sym(const double *__restrict__ U, int n, int i,
                                            const double (&v)[10]) {
    const double2 z2 = make_double2(0.0, 0.0);
    if (!AIRGA_CK(i, 0, n - 1, 103)) return z2;
    const double2 *U0 = reinterpret_cast<const double2 *>(U);
    const double2 *U1 = reinterpret_cast<const double2 *>(U + n);
    const double2 *U2 = reinterpret_cast<const double2 *>(U + 2 * (long long)n);
    const double2 *U3 = reinterpret_cast<const double2 *>(U + 3 * (long long)n);
    const int h = i >> 1;                                   // double2 index of rows (i, i+1)
    const double2 u0 = __ldg(U0 + h), u1 = __ldg(U1 + h), u2 = __ldg(U2 + h), u3 = __ldg(U3 + h);
    const double2 l1 = i >= 2 ? __ldg(U1 + h - 1) : z2;     // U1[i-2], U1[i-1]
    const double2 l2 = i >= 2 ? __ldg(U2 + h - 1) : z2;     // U2[i-2], U2[i-1]
    const double2 l3a = i >= 4 ? __ldg(U3 + h - 2) : z2;    // U3[i-4], U3[i-3]
    const double2 l3b = i >= 2 ? __ldg(U3 + h - 1) : z2;    // U3[i-2], U3[i-1]
    double y0 = l3a.y * v[1];
    y0 = fma(l2.x, v[2], y0);
    y0 = fma(l1.y, v[3], y0);
    y0 = fma(u0.x, v[4], y0);
    y0 = fma(u1.x, v[5], y0);
    y0 = fma(u2.x, v[6], y0);
    y0 = fma(u3.x, v[7], y0);
    double y1 = l3b.x * v[2];
    y1 = fma(l2.y, v[3], y1);
    y1 = fma(u1.x, v[4], y1);
    y1 = fma(u0.y, v[5], y1);
    y1 = fma(u1.y, v[6], y1);
    y1 = fma(u2.y, v[7], y1);
    y1 = fma(u3.y, v[8], y1);
    return make_double2(y0, y1);
}

// Same with the beam's exact zeros skipped: even row drops d = 0 (-3) and
// d = 4 (+1); odd row drops d = 6 (+3) and d = 2 (-1).  The free-end pair
// (i = n-2) keeps its +-1 couplings.
__device__ __forceinline__ double2 pair_beam(const double2 (&a)[kBand], const double (&v)[10],
                                             bool last) {
    double y0 = a[1].x * v[2];
    y0 = fma(a[2].x, v[3], y0);
    y0 = fma(a[3].x, v[4], y0);
    y0 = fma(a[5].x, v[6], y0);
    y0 = fma(a[6].x, v[7], y0);
    double y1 = a[0].y * v[2];
    y1 = fma(a[1].y, v[3], y1);
    y1 = fma(a[3].y, v[5], y1);
    y1 = fma(a[4].y, v[6], y1);
    y1 = fma(a[5].y, v[7], y1);
    if (last) {
        y0 = fma(a[4].x, v[5], y0);
        y1 = fma(a[2].y, v[4], y1);
    }
    return make_double2(y0, y1);
}

// Warm L2 with the 16-byte rows of `count` band arrays of stride n at pair i
// (no registers held; issued before a barrier so the first loads of the next
// phase find their lines in L2 instead of DRAM).
__device__ __forceinline__ void prefetch_pair(const double *band, int n, int i, int count) {
    for (int k = 0; k < count; ++k)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(band + (long long)k * n + i));
}

// Beam row pair from the packed nonzeros (5 double2 loads = 80 B instead of
// the band's 112 B): even row offsets (-2,-1,0,+2,+3), odd row
// (-3,-2,0,+1,+2); the free-end pair adds its +-1 couplings from the band.
__device__ __forceinline__ void load_packed(const double *__restrict__ pk, int n, int i,
                                            double2 (&c)[5]) {
    if (!AIRGA_CK(i, 0, n - 1, 104)) {
#pragma unroll
        for (int k = 0; k < 5; ++k) c[k] = make_double2(0.0, 0.0);
        return;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) c[k] = __ldg(reinterpret_cast<const double2 *>(pk + (long long)k * n + i));
}

__device__ __forceinline__ double2 pair_packed_c(const double2 (&c)[5],
                                                 const double *__restrict__ band, int n,
                                                 int i, const double (&v)[10]) {
    double y0 = c[0].x * v[2];
    y0 = fma(c[1].x, v[3], y0);
    y0 = fma(c[2].x, v[4], y0);
    y0 = fma(c[3].x, v[6], y0);
    y0 = fma(c[4].x, v[7], y0);
    double y1 = c[0].y * v[2];
    y1 = fma(c[1].y, v[3], y1);
    y1 = fma(c[2].y, v[5], y1);
    y1 = fma(c[3].y, v[6], y1);
    y1 = fma(c[4].y, v[7], y1);
    if (i == n - 2) {
        y0 = fma(__ldg(band + 4LL * n + i), v[5], y0);
        y1 = fma(__ldg(band + 2LL * n + i + 1), v[4], y1);
    }
    return make_double2(y0, y1);
}

// Right-hand side row i: b_i, or rhs_scale (M v)_i when the RHS is formed
// on the fly from a band matrix M and a vector v (the AIRGA inner-loop
// right-hand sides M V_j, Alg. 3 / Alg. 5), so M V is never stored.
__device__ __forceinline__ double rhs_row(const PcgArgs &a, int n, int i) {
    if (!AIRGA_CK(i, 0, n, 105)) return 0.0;
    if (!a.rhs_M) return a.b[i];
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < kBand; ++d) {
        const int c = i + d - kHalf;
        if (c >= 0 && c < n) acc = fma(__ldg(a.rhs_M + (long long)d * n + i), __ldg(a.rhs_v + c), acc);
    }
    return a.rhs_scale * acc;
}

// Block-wide scalars of one solve.
struct PairShared {
    double tot[8];
    int s_flag;
    int s_dec;
    double s_nb;
};

// The whole solve of one system by one CTA of a group of G CTAs, this CTA
// being `rank` (rows [rank R, rank R + R)).  The group's barriers, partials
// and p boundary buffer come from `a`; the single-system kernel runs it with
// the whole grid as the group, the batched kernel once per assignment.
// SYMU: read P_sym through its upper diagonals (pair_sym; every kernel that
// has P_sym does)
// SLOT_SLICE (batch lanes): a.state is this CTA's own z/q slice, not the base
// of the group's slices
template <int MODE, int SPLIT = 0, bool SYMU = true, bool SLOT_SLICE = false>   // MODE 0: identity, 1: one symmetric band
__device__ void pair_body(const PcgArgs &a, int R, int G, int rank, double *smem,
                          PairShared &sh) {
    double *tot = sh.tot;
    int &s_flag = sh.s_flag;
    int &s_dec = sh.s_dec;
    double &s_nb = sh.s_nb;
    const int n = (int)a.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lo = rank * R < n ? rank * R : n;
    const int hi = lo + R < n ? lo + R : n;
    if (tid == 0) s_nb = 0.0;
    if (a.place && tid == 0) {                     // test hook: where this CTA runs
        unsigned sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        a.place[rank] = (int32_t)sm;
    }

    // SPLIT == 0: x, r, p, z/q windows all in shared memory.  SPLIT == 1 (n too
    // large for four windows) and SPLIT == 2 (half an SM per CTA): r and p
    // stay in shared memory, x is updated in place in the caller's X and the
    // z/q window lives in this CTA's slice of the global workspace (L2
    // traffic of 48 B per row and iteration).
    double *xs, *rs, *ps, *zq;
    if (SPLIT) {
        rs = smem;
        ps = rs + (R + 2 * HR);
        xs = a.x + lo;
        zq = a.state + (SLOT_SLICE ? (size_t)0 : (size_t)rank * (size_t)(R + 2 * HZ));
    } else {
        xs = smem;
        rs = xs + R;
        ps = rs + (R + 2 * HR);
        zq = ps + (R + 2 * HZ);
    }
    double2 *ah = reinterpret_cast<double2 *>(ps + (R + 2 * HZ) + (SPLIT ? 0 : R + 2 * HZ));   // A rows of the r halo
    double *red = reinterpret_cast<double *>(ah + kHaloPairs * kBand);
    const int xbase = lo, rbase = lo - HR, pbase = lo - HZ, zbase = lo - HZ;
    const int lenR = R + 2 * HR, lenZ = R + 2 * HZ;      // window lengths (r; p and z/q)
    (void)lenR;
    (void)lenZ;
    const int rlo = lo - HR > 0 ? lo - HR : 0, rhi = hi + HR < n ? hi + HR : n;
    const int zlo = lo - HZ > 0 ? lo - HZ : 0, zhi = hi + HZ < n ? hi + HZ : n;
    const int bw = HP < (hi - lo) ? HP : (hi - lo);
    const bool beam = a.pairz != nullptr && *a.pairz != 0;
    const bool packed = beam && a.Apk != nullptr;
    const double *Pb = MODE == 1 ? (a.psym ? a.psym : a.fac[0]) : nullptr;
    // P_sym is symmetric: read its upper diagonals only (rows 3n.. of the band)
    const double *Psu = SYMU && MODE == 1 && a.psym ? a.psym + 3 * (long long)n : nullptr;
    // r-halo pairs are recomputed by the last kHaloPairs threads (they own
    // one pair fewer than the first threads when R/2 is not a multiple of nt)
    const int hslot = nt - 1 - tid;                  // 0..7 for the halo threads
    const bool halo_thread = hslot < kHaloPairs;
    const int hpair = hslot < kHaloPairs / 2 ? lo - HR + 2 * hslot
                                                 : hi + 2 * (hslot - kHaloPairs / 2);
    const bool hvalid = halo_thread && hpair >= 0 && hpair < n;

    // zero every window (out-of-matrix slots must read as 0), cache A's halo rows
    {
        const int total = SPLIT ? 2 * R + 2 * (HR + HZ) : 4 * R + 2 * (HR + 2 * HZ);
        for (int k = tid; k < total; k += nt) smem[k] = 0.0;
        if (SPLIT)
            for (int k = tid; k < R + 2 * HZ; k += nt) zq[k] = 0.0;
        if (hvalid) {
            double2 t[kBand];
            load_band_pair(a.A, n, hpair, t);
#pragma unroll
            for (int d = 0; d < kBand; ++d) ah[hslot * kBand + d] = t[d];
        }
    }
    __syncthreads();

    unsigned bar_no = 0;
    const long long tmo = a.timeout_ns;
    int status = AIRGA_E_MAXIT;
    int iters = 0;

    // ---- x_0, r_0 = b - A x_0 on own +- HR, z_0 = M r_0 on own +- HZ ----
    for (int i = lo + tid; i < hi; i += nt) xs[i - xbase] = a.warm ? a.x[i] : 0.0;
    for (int i = rlo + tid; i < rhi; i += nt) {
        double v = rhs_row(a, n, i);
        if (a.warm) {
            double ax = 0.0;
#pragma unroll
            for (int d = 0; d < kBand; ++d) {
                const int c = i + d - kHalf;
                if (c >= 0 && c < n) ax = fma(__ldg(a.A + (long long)d * n + i), a.x[c], ax);
            }
            v -= ax;
        }
        rs[i - rbase] = v;
    }
    __syncthreads();
    // z = M r for the pairs [from, to) (stride 2 nt starting at this thread's
    // slot); r.z and r.r of own pairs accumulate into v2
    auto apply_M = [&](int from, int to, double (&v2)[2]) {
        for (int i = from + 2 * tid; i < to; i += 2 * nt) {
            double2 z;
            if (MODE == 1 && Psu) {
                double v[10];
                load_win(rs, rbase, i, v, lenR);
                z = pair_sym(Psu, n, i, v);
            } else if (MODE == 1) {
                double2 pb[kBand];
                load_band_pair(Pb, n, i, pb);
                double v[10];
                load_win(rs, rbase, i, v, lenR);
                z = pair_full(pb, v);
            } else {
                z = AIRGA_CK(i - rbase, 0, lenR - 1, 106)
                        ? *reinterpret_cast<const double2 *>(rs + (i - rbase))
                        : make_double2(0.0, 0.0);
            }
            if (AIRGA_CK(i - zbase, 0, lenZ - 1, 107))
                *reinterpret_cast<double2 *>(zq + (i - zbase)) = z;
            if (i >= lo && i < hi) {
                const double2 r = *reinterpret_cast<const double2 *>(rs + (i - rbase));
                v2[0] = fma(r.x, z.x, fma(r.y, z.y, v2[0]));
                v2[1] = fma(r.x, r.x, fma(r.y, r.y, v2[1]));
            }
        }
    };
    {
        double v2[2] = {0.0, 0.0};
        apply_M(zlo, zhi, v2);
        double v[3] = {v2[0], v2[1], 0.0};
        for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
            if (a.rhs_M) {
                // b = c M v formed in the kernel: with x_0 = 0 the r_0 window
                // already holds it (no second band product)
                const double b0 = a.warm ? rhs_row(a, n, i) : rs[i - rbase];
                const double b1 = a.warm ? rhs_row(a, n, i + 1) : rs[i + 1 - rbase];
                v[2] = fma(b0, b0, fma(b1, b1, v[2]));
            } else {
                const double2 b = *reinterpret_cast<const double2 *>(a.b + i);
                v[2] = fma(b.x, b.x, fma(b.y, b.y, v[2]));
            }
        }
        block_partials_tree<3>(v, red, a.partials, bar_no & 1, G, rank);
    }
    if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag, true, G)) {
        status = AIRGA_E_TIMEOUT;
        goto finish;
    }
    double t0[3];
    grid_totals<3>(a.partials, bar_no & 1, G, tot, t0);
    ++bar_no;
    {
        double rz = t0[0];
        const double bb = t0[2];
        const double nb = sqrt(bb);
        const double thr2 = (a.tol * nb) * (a.tol * nb);     // stop when r.r <= (tol ||b||)^2
        if (tid == 0) s_nb = nb;
        if (rank == 0 && tid == 0 && a.hist) a.hist[0] = t0[1];
        if (nb == 0.0) {
            for (int i = lo + tid; i < hi; i += nt) xs[i - xbase] = 0.0;
            status = AIRGA_OK;
            goto finish;
        }
        if (t0[1] <= thr2) { status = AIRGA_OK; goto finish; }
        if (!isfinite(rz) || rz == 0.0) { status = AIRGA_E_BREAKDOWN; goto finish; }

        double beta = 0.0;
        for (int k = 1; k <= a.maxit; ++k) {
            // ---- phase 1: p = z + beta p on own +- 4; boundary rows out; q = A p ----
            for (int i = zlo + 2 * tid; i < zhi; i += 2 * nt) {
                if (!AIRGA_CK(i - pbase, 0, lenZ - 1, 108)) continue;
                double2 *pp = reinterpret_cast<double2 *>(ps + (i - pbase));
                const double2 z = *reinterpret_cast<const double2 *>(zq + (i - zbase));
                if (k == 1) {
                    *pp = z;
                } else {
                    double2 p = *pp;
                    p.x = fma(beta, p.x, z.x);
                    p.y = fma(beta, p.y, z.y);
                    *pp = p;
                }
            }
            __syncthreads();
            for (int t = tid; t < 2 * bw; t += nt) {
                const int i = t < bw ? lo + t : hi - bw + (t - bw);
                if (AIRGA_CK(i, 0, n, 109) && AIRGA_CK(i - pbase, 0, lenZ, 110))
                    a.pbuf[i] = ps[i - pbase];
            }
            double vq[1] = {0.0};
            if (packed) {
                for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
                    double2 c[5];
                    load_packed(a.Apk, n, i, c);
                    double v[10];
                    load_win(ps, pbase, i, v, lenZ);
                    const double2 q = pair_packed_c(c, a.A, n, i, v);
                    if (AIRGA_CK(i - zbase, 0, lenZ - 1, 111))
                        *reinterpret_cast<double2 *>(zq + (i - zbase)) = q;
                    vq[0] = fma(v[4], q.x, fma(v[5], q.y, vq[0]));
                }
            } else {
                for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
                    double2 ab[kBand];
                    load_band_pair(a.A, n, i, ab);
                    double v[10];
                    load_win(ps, pbase, i, v, lenZ);
                    const double2 q = beam ? pair_beam(ab, v, i == n - 2) : pair_full(ab, v);
                    if (AIRGA_CK(i - zbase, 0, lenZ - 1, 112))
                        *reinterpret_cast<double2 *>(zq + (i - zbase)) = q;
                    vq[0] = fma(v[4], q.x, fma(v[5], q.y, vq[0]));
                }
            }
            if (MODE == 1 && zlo + 2 * tid < zhi) {
                if (Psu) prefetch_pair(Psu, n, zlo + 2 * tid, 4);
                else prefetch_pair(Pb, n, zlo + 2 * tid, kBand);
            }
            block_partials_tree<1>(vq, red, a.partials, bar_no & 1, G, rank);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag, true, G)) {
                status = AIRGA_E_TIMEOUT;
                iters = k - 1;
                goto finish;
            }
            // warp 0: (p, q) total, breakdown test and alpha; one CTA barrier
            if (tid < 32) {
                double pqt[1];
                warp0_totals<1>(a.partials, bar_no & 1, G, pqt);
                if (tid == 0) {
                    const double pq = pqt[0];
                    const bool bad = !(pq > 0.0) || !isfinite(pq);
                    s_dec = bad ? 1 : 0;
                    tot[0] = bad ? 0.0 : rz * lean::rcp_signed(pq);
                }
            }
            __syncthreads();
            ++bar_no;
            if (s_dec) {
                status = AIRGA_E_BREAKDOWN;
                iters = k - 1;
                goto finish;
            }
            const double alpha = tot[0];

            // ---- phase 2: x, r updates; r halo (beside the x/r sweep); z = M r ----
            double pv[10];
            if (hvalid) {
                // p around this halo pair: the outer rows come from their owners
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    const int row = hpair - 4 + q;
                    double v = 0.0;
                    if (row >= 0 && row < n)
                        v = (row >= lo - HZ && row < hi + HZ) ? ps[row - pbase] : __ldcg(a.pbuf + row);
                    pv[q] = v;
                }
            }
            for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
                if (!AIRGA_CK(i - xbase, 0, R - 1, 113) || !AIRGA_CK(i - rbase, 0, lenR - 1, 114))
                    continue;
                double2 *xp = reinterpret_cast<double2 *>(xs + (i - xbase));
                double2 *rp = reinterpret_cast<double2 *>(rs + (i - rbase));
                const double2 p = *reinterpret_cast<const double2 *>(ps + (i - pbase));
                const double2 q = *reinterpret_cast<const double2 *>(zq + (i - zbase));
                double2 x = *xp, r = *rp;
                x.x = fma(alpha, p.x, x.x);
                x.y = fma(alpha, p.y, x.y);
                r.x = fma(-alpha, q.x, r.x);
                r.y = fma(-alpha, q.y, r.y);
                *xp = x;
                *rp = r;
            }
            if (hvalid) {
                // the r halo needs no own-row update: it runs beside the x/r sweep
                double2 t[kBand];
#pragma unroll
                for (int d = 0; d < kBand; ++d) t[d] = ah[hslot * kBand + d];
                const double2 q = beam ? pair_beam(t, pv, hpair == n - 2) : pair_full(t, pv);
                if (AIRGA_CK(hpair - rbase, 0, lenR - 1, 115)) {
                    double2 *rp = reinterpret_cast<double2 *>(rs + (hpair - rbase));
                    double2 r = *rp;
                    r.x = fma(-alpha, q.x, r.x);
                    r.y = fma(-alpha, q.y, r.y);
                    *rp = r;
                }
            }
            __syncthreads();
            double v2[2] = {0.0, 0.0};
            apply_M(zlo, zhi, v2);
            if (lo + 2 * tid < hi) {
                if (packed) prefetch_pair(a.Apk, n, lo + 2 * tid, 5);
                else prefetch_pair(a.A, n, lo + 2 * tid, kBand);
            }
            block_partials_tree<2>(v2, red, a.partials, bar_no & 1, G, rank);
            const bool arrive = !(a.fault_skip_arrival && k == 1 && rank == 0);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag,
                              arrive, G)) {
                status = AIRGA_E_TIMEOUT;
                iters = k;
                goto finish;
            }
            // warp 0: (r, z) and (r, r) totals, stopping tests and beta
            if (tid < 32) {
                double t2v[2];
                warp0_totals<2>(a.partials, bar_no & 1, G, t2v);
                if (tid == 0) {
                    if (rank == 0 && a.hist) a.hist[k] = t2v[1];
                    const double rz_new = t2v[0];
                    int dec = 0;
                    if (t2v[1] <= thr2) dec = 1;                               // converged
                    else if (!isfinite(rz_new) || rz_new == 0.0) dec = 2;      // breakdown
                    s_dec = dec;
                    tot[1] = dec ? 0.0 : rz_new * lean::rcp_signed(rz);        // beta
                    tot[2] = rz_new;
                }
            }
            __syncthreads();
            ++bar_no;
            iters = k;
            {
                const int dec = s_dec;
                if (dec == 1) { status = AIRGA_OK; break; }
                if (dec == 2) { status = AIRGA_E_BREAKDOWN; break; }
            }
            beta = tot[1];
            rz = tot[2];
        }
    }
finish:
    __syncthreads();
    if (!SPLIT)
        for (int i = lo + tid; i < hi; i += nt) a.x[i] = xs[i - xbase];
    if (rank == 0) {
        if (a.hist && s_nb > 0.0)       // r.r -> ||r_k|| / ||b||
            for (int k = tid; k <= iters; k += nt) a.hist[k] = sqrt(a.hist[k]) / s_nb;
        if (tid == 0) {
            if (a.hist && !(s_nb > 0.0)) a.hist[0] = 0.0;
            *a.iters = iters;
            *a.status = status;
        }
    }
    if (a.relres && status == AIRGA_E_TIMEOUT && rank == 0 && tid == 0)
        *a.relres = __longlong_as_double(0x7FF8000000000000ll);   // NaN: no residual pass after an abort
    if (a.relres && status != AIRGA_E_TIMEOUT) {
        // true residual ||b - A x|| / ||b|| of the final x, in FP64: the group
        // exchanges x through global memory (one barrier), each CTA sums its rows
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag, true, G)) return;
        ++bar_no;
        double v[2] = {0.0, 0.0};
        for (int i = lo + tid; i < hi; i += nt) {
            double ax = 0.0;
#pragma unroll
            for (int d = 0; d < kBand; ++d) {
                const int c = i + d - kHalf;
                if (c >= 0 && c < n) ax = fma(__ldg(a.A + (long long)d * n + i), __ldcg(a.x + c), ax);
            }
            const double bi = rhs_row(a, n, i), r = bi - ax;
            v[0] = fma(r, r, v[0]);
            v[1] = fma(bi, bi, v[1]);
        }
        block_partials_tree<2>(v, red, a.partials, bar_no & 1, G, rank);
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag, true, G)) return;
        if (rank == 0 && tid < 32) {
            double t[2];
            warp0_totals<2>(a.partials, bar_no & 1, G, t);
            if (tid == 0) *a.relres = t[1] > 0.0 ? sqrt(t[0]) / sqrt(t[1]) : 0.0;
        }
    }
}

template <int MODE, int SPLIT>
__global__ void __launch_bounds__(SPLIT == 2 ? kThreadsHalf : (SPLIT ? kThreadsSplit : kThreadsFull),
                                  SPLIT == 2 ? 2 : 1)
pcg_pair_kernel(PcgArgs a, int R) {
    extern __shared__ __align__(16) double smem[];
    __shared__ PairShared sh;
    pair_body<MODE, SPLIT>(a, R, gridDim.x, blockIdx.x, smem, sh);
}

// Batched form: CTA c runs the assignments asg[off[c] .. off[c+1]) in order;
// each names a system (its PcgArgs in `sys`, with group-private barrier,
// partials and p buffer), the group size, this CTA's rank and the rows per
// CTA.  Assignments are appended in one global order of systems, so a CTA
// waiting at a group barrier only waits for CTAs that are at the same or an
// earlier system in that order: the schedule cannot deadlock.
//
// LANES (options.sm_share 2 or 3): two lanes of gridDim.x / 2 CTA slots,
// two CTAs per SM (256 threads, half an SM each, r and p windows in shared
// memory, x in place, z/q in the slot's own global slice).  A CTA takes its
// lane from its arrival on its SM (first: lane 0, second: lane 1; a full lane
// sends it to the other), so every SM holds one CTA of each lane, and the
// systems of the two lanes fill each other's barrier gaps.  Each system's
// group lies within one lane; each lane's lists follow one global order.
// roles: [0], [1] lane counters, [2 + s] arrivals on SM s (zeroed per solve).
template <int MODE, int LANES>
__global__ void __launch_bounds__(LANES ? kThreadsHalf : kThreadsBatch, LANES ? 2 : 1)
pcg_pair_batch_kernel(const PcgArgs *__restrict__ sys, const int4 *__restrict__ asg,
                      const int *__restrict__ off, unsigned *roles, double *slices,
                      int slice_len) {
    extern __shared__ __align__(16) double smem[];
    __shared__ PairShared sh;
    __shared__ int s_slot;
    int slot = blockIdx.x;
    if (LANES) {
        const int L = (int)(gridDim.x / 2);
        if (threadIdx.x == 0) {
            unsigned sm;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
            int lane = (int)(atomicAdd(&roles[2 + (sm & 1023u)], 1u) & 1u);
            unsigned r = atomicAdd(&roles[lane], 1u);
            if ((int)r >= L) {
                lane ^= 1;
                r = atomicAdd(&roles[lane], 1u);
            }
            s_slot = lane * L + (int)r;
        }
        __syncthreads();
        slot = s_slot;
        if (!AIRGA_CK(slot, 0, 2 * L, 116)) return;
    }
    const int b = off[slot], e = off[slot + 1];
    for (int k = b; k < e; ++k) {
        const int4 w = asg[k];                       // (system, group size, rank, rows per CTA)
        PcgArgs a = sys[w.x];
        if ((MODE == 1) == (a.nf == 1)) {
            if (LANES) {
                a.state = slices + (size_t)slot * (size_t)slice_len;
                pair_body<MODE, 2, true, true>(a, w.w, w.y, w.z, smem, sh);
            } else {
                pair_body<MODE, 0, true>(a, w.w, w.y, w.z, smem, sh);
            }
        }
        __syncthreads();
    }
}

template <int MODE, int SPLIT>
cudaError_t launch_pair_mode(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s) {
    auto kern = pcg_pair_kernel<MODE, SPLIT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem_bytes);
    if (e != cudaSuccess) return e;
    if (SPLIT == 2) {
        // the SMs must be configured for the largest shared-memory carveout:
        // a lead CTA alone would otherwise get a smaller one (more L1), and a
        // partner CTA would find no room beside it
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    PcgArgs a = args;
    int R = (int)plan.rows;
    void *kargs[] = {(void *)&a, (void *)&R};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(plan.grid), dim3(plan.threads),
                                       kargs, plan.smem_bytes, s);
}

}  // namespace

size_t pcg_pair_smem(int64_t R) {
    return (size_t)(4 * R + 2 * (HR + 2 * HZ) + 2 * kHaloPairs * kBand + 3 * kThreadsMax) *
           sizeof(double);
}

size_t pcg_pair_split_smem(int64_t R) {
    return (size_t)(2 * R + 2 * (HR + HZ) + 2 * kHaloPairs * kBand + 3 * kThreadsSplit) * sizeof(double);
}

size_t pcg_pair_half_smem(int64_t R) {
    return (size_t)(2 * R + 2 * (HR + HZ) + 2 * kHaloPairs * kBand + 3 * kThreadsHalf) * sizeof(double);
}

size_t pcg_pair_split_slice(int64_t R) { return (size_t)(R + 2 * HZ); }

int pcg_pair_threads(int kind) {
    return kind == 3 ? kThreadsSplit : (kind == 4 ? kThreadsHalf : kThreadsFull);
}

size_t pcg_pair_half_static_smem(int mode) {
    cudaFuncAttributes fa;
    const void *kern = mode == 0 ? (const void *)pcg_pair_kernel<0, 2> : (const void *)pcg_pair_kernel<1, 2>;
    return cudaFuncGetAttributes(&fa, kern) == cudaSuccess ? fa.sharedSizeBytes : 256;
}

int pcg_pair_half_occupancy(int mode, size_t smem, int *per_sm) {
    const void *kern = mode == 0 ? (const void *)pcg_pair_kernel<0, 2> : (const void *)pcg_pair_kernel<1, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, kThreadsHalf, smem);
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "pcg pair half occupancy");
}

int pcg_pair_occupancy(int mode, size_t smem, int *per_sm) {
    cudaError_t e;
    if (mode == 0) {
        e = cudaFuncSetAttribute(pcg_pair_kernel<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pcg_pair_kernel<0, 0>, kThreadsFull, smem);
    } else {
        e = cudaFuncSetAttribute(pcg_pair_kernel<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pcg_pair_kernel<1, 0>, kThreadsFull, smem);
    }
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "pcg pair occupancy");
}

static const void *batch_kernel(int mode, bool half) {
    if (half)
        return mode ? (const void *)pcg_pair_batch_kernel<1, 1> : (const void *)pcg_pair_batch_kernel<0, 1>;
    return mode ? (const void *)pcg_pair_batch_kernel<1, 0> : (const void *)pcg_pair_batch_kernel<0, 0>;
}

int pcg_pair_batch_threads(bool half) { return half ? kThreadsHalf : kThreadsBatch; }

size_t pcg_pair_batch_smem(int64_t R, bool half) {
    if (half) return pcg_pair_half_smem(R);                 // lanes: the split state
    return (size_t)(4 * R + 2 * (HR + 2 * HZ) + 2 * kHaloPairs * kBand + 3 * kThreadsBatch) *
           sizeof(double);
}

size_t pcg_pair_batch_slice(int64_t R) { return (size_t)(R + 2 * HZ); }

size_t pcg_pair_batch_static_smem(bool half) {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, batch_kernel(1, half)) == cudaSuccess ? fa.sharedSizeBytes : 256;
}

int pcg_pair_batch_prepare(int mode, size_t smem, bool half) {
    const void *kern = batch_kernel(mode, half);
    cudaError_t e = cudaSuccess;
    if (half)   // two CTAs per SM need the largest shared-memory carveout
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "batch smem");
}

int pcg_pair_batch_occupancy(int mode, size_t smem, int *per_sm, bool half) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel(mode, half),
                                                                  pcg_pair_batch_threads(half), smem);
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "batch occupancy");
}

cudaError_t launch_pcg_pair_batch(int mode, int grid, size_t smem, const PcgArgs *sys,
                                  const int4 *asg, const int *off, bool half, unsigned *roles,
                                  double *slices, int slice_len, cudaStream_t s) {
    void *kargs[] = {(void *)&sys, (void *)&asg, (void *)&off, (void *)&roles, (void *)&slices,
                     (void *)&slice_len};
    return cudaLaunchCooperativeKernel(batch_kernel(mode, half), dim3(grid),
                                       dim3(pcg_pair_batch_threads(half)), kargs, smem, s);
}

int pcg_pair_split_occupancy(int mode, size_t smem, int *per_sm) {
    cudaError_t e;
    if (mode == 0) {
        e = cudaFuncSetAttribute(pcg_pair_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pcg_pair_kernel<0, 1>, kThreadsSplit, smem);
    } else {
        e = cudaFuncSetAttribute(pcg_pair_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pcg_pair_kernel<1, 1>, kThreadsSplit, smem);
    }
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "pcg pair split occupancy");
}

cudaError_t launch_pcg_pair(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s) {
    if (plan.kind == 4) {
        if (args.nf == 0) return launch_pair_mode<0, 2>(plan, args, s);
        return launch_pair_mode<1, 2>(plan, args, s);
    }
    if (plan.kind == 3) {
        if (args.nf == 0) return launch_pair_mode<0, 1>(plan, args, s);
        return launch_pair_mode<1, 1>(plan, args, s);
    }
    if (args.nf == 0) return launch_pair_mode<0, 0>(plan, args, s);
    return launch_pair_mode<1, 0>(plan, args, s);
}

}  // namespace airga

AIRGA_CHECK_READER(pcg_pair)

// ---------------------------------------------------------------------------
// Stream hold for lead / partner solves (options.sm_share 2 and 3): one warp
// that sleeps for a bounded time on the global timer.  Queued on the
// partners' stream right after the lead's inputs are ready, it keeps partner
// work off the SMs while the lead's CTAs are dispatched (a cooperative grid
// is placed CTA by CTA; an SM taken by partner work at that moment would
// leave one lead CTA waiting for it at the lead's first barrier).
// ---------------------------------------------------------------------------
namespace airga {
namespace {
// Sleeps until the global timer has advanced `ns`; the loop is also capped at
// `ns` rounds (each round takes well over a nanosecond), so it ends even if
// the timer were to stall.
__global__ void stream_hold_kernel(long long ns) {
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (long long round = 0; round < ns; ++round) {
        __nanosleep(1000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) >= ns) break;
    }
}
}  // namespace
}  // namespace airga

extern "C" int airga_stream_hold(int32_t microseconds, void *stream) {
    if (microseconds < 0 || microseconds > 1000)
        return airga::fail(AIRGA_E_INVALID_ARG, "microseconds must be in [0, 1000]");
    if (microseconds == 0) return AIRGA_OK;
    airga::stream_hold_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)microseconds * 1000);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AIRGA_OK : airga::cuda_fail(e, "stream hold");
}
