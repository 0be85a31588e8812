// Mixed precision: FP32 inner preconditioned CG inside FP64 iterative
// refinement (airga_pcg_solve_mixed).
//
// Per right-hand side f, with x = 0:
//   k = 0, 1, ...:  r = f - A x            FP64 (true residual)
//                   stop if ||r|| <= tol ||f||  (or after max_outer steps)
//                   A d = r by FP32 PCG   (FP32 bands of A and P_sym, FP32
//                                          vectors, d_0 = 0)
//                   x = x + d             FP64
// One persistent launch per column runs the whole loop: the FP64 residual of
// a CTA's rows (and of its r-halo rows) goes straight into its FP32 residual
// window, the convergence test is a grid reduction, and the update of x is
// followed by a grid barrier so the next residual sees the neighbours' rows.
// A column therefore costs one launch however many steps it takes, and none
// is spent on steps that are never needed.
//
// Why on GB300: an FP64 FMA issues at 2/clk/SM, an FP32 FMA at 128/clk/SM.
// The inner iterations — the bulk of the work — leave the FP64 pipe for the
// FP32 one and halve the band and vector bytes (FP32 copies of A and P_sym
// stay resident in L2 up to n of about 2.3e6); FP64 is kept where accuracy
// is decided: the outer residual, the refinement update, the SPAI QR, and
// the grid totals and step lengths of the inner CG.  Each CTA sums its
// threads' FP32 partials in FP32 (a tree of FP32 adds instead of FP64 ones,
// whose latency the otherwise idle inner loop would wait on); the 152 CTA
// sums are added in FP64.
//
// The inner solve is the row-pair persistent PCG of pcg_pair.cu with float
// data: same ownership, halo and barrier scheme, r halo recomputed beside
// the x/r sweep, warp-0 scalar updates.
#include "check.cuh"
#include "fp64_lean.cuh"
#include "pcg_common.cuh"

namespace airga {
namespace {

using namespace pcgdev;

constexpr int kThreads = 512;
constexpr int HR = 8, HP = 12, HZ = 4, kHaloPairs = 8;

// ---------------------------------------------------------------------------
// FP64 -> FP32 copies
// ---------------------------------------------------------------------------
__global__ void to_f32_kernel(int64_t total, const double *__restrict__ src,
                              float *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// ---------------------------------------------------------------------------
// The refinement loop of one column (FP64 residual, FP32 row-pair PCG)
// ---------------------------------------------------------------------------
struct Args32 {
    int n;
    const float *A;       // FP32 band-7 of A
    const float *Apk;     // FP32 packed beam nonzeros of A, or null
    const int32_t *pairz; // beam structure flag of A (device), or null
    const float *M;       // FP32 band-7 preconditioner (or null = identity)
    const double *A64;    // FP64 band-7 of A (outer residual)
    const double *f;      // right-hand side column
    double *x64;          // refinement iterate (zeroed by the kernel)
    float *pbuf;
    double *partials;
    unsigned *bar;
    int *abort_flag;
    double tol;           // outer (FP64) relative tolerance
    double inner_tol;     // inner relative tolerance
    int maxit;            // inner iterations per refinement step
    int max_outer;        // refinement steps
    long long timeout_ns;
    int fault_skip_arrival; // test hook: CTA 0 skips its first inner barrier arrival
    double *relres;       // out: FP64 relative residual at exit
    int32_t *outer_iters; // out: refinement steps taken
    int32_t *inner_iters; // out: FP32 CG iterations, all steps
    int32_t *status;      // out
};

// Warm L2 with the 8-byte rows of `count` FP32 band arrays at pair i (no
// registers held; issued before a barrier so the next phase's first loads
// find their lines in L2).
__device__ __forceinline__ void prefetch_pair_f(const float *band, int n, int i, int count) {
    for (int k = 0; k < count; ++k)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(band + (long long)k * n + i));
}

__device__ __forceinline__ void load_band_pair_f(const float *__restrict__ band, int n, int i,
                                                 float2 (&a)[kBand]) {
    if (!AIRGA_CK(i, 0, n - 1, 601)) {
#pragma unroll
        for (int d = 0; d < kBand; ++d) a[d] = make_float2(0.0f, 0.0f);
        return;
    }
#pragma unroll
    for (int d = 0; d < kBand; ++d)
        a[d] = __ldg(reinterpret_cast<const float2 *>(band + (long long)d * n + i));
}

// wlen: the window's length (checked builds test the ten rows against it)
__device__ __forceinline__ void load_win_f(const float *w, int wbase, int i, float (&v)[10],
                                           int wlen) {
    if (!AIRGA_CK(i - 4 - wbase, 0, wlen - 9, 602)) {
#pragma unroll
        for (int k = 0; k < 10; ++k) v[k] = 0.0f;
        return;
    }
    const float2 *w2 = reinterpret_cast<const float2 *>(w + (i - 4 - wbase));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float2 t = w2[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ float2 pair_full_f(const float2 (&a)[kBand], const float (&v)[10]) {
    float y0 = a[0].x * v[1], y1 = a[0].y * v[2];
#pragma unroll
    for (int d = 1; d < kBand; ++d) {
        y0 = fmaf(a[d].x, v[1 + d], y0);
        y1 = fmaf(a[d].y, v[2 + d], y1);
    }
    return make_float2(y0, y1);
}

// packed beam pair (see pack_pairs in band_kernels.cu), free-end couplings from the band
__device__ __forceinline__ float2 pair_packed_f(const float *__restrict__ pk,
                                                const float *__restrict__ band, int n, int i,
                                                const float (&v)[10]) {
    float2 c[5];
    if (!AIRGA_CK(i, 0, n - 1, 603)) return make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 5; ++k) c[k] = __ldg(reinterpret_cast<const float2 *>(pk + (long long)k * n + i));
    float y0 = c[0].x * v[2];
    y0 = fmaf(c[1].x, v[3], y0);
    y0 = fmaf(c[2].x, v[4], y0);
    y0 = fmaf(c[3].x, v[6], y0);
    y0 = fmaf(c[4].x, v[7], y0);
    float y1 = c[0].y * v[2];
    y1 = fmaf(c[1].y, v[3], y1);
    y1 = fmaf(c[2].y, v[5], y1);
    y1 = fmaf(c[3].y, v[6], y1);
    y1 = fmaf(c[4].y, v[7], y1);
    if (i == n - 2) {
        y0 = fmaf(__ldg(band + 4LL * n + i), v[5], y0);
        y1 = fmaf(__ldg(band + 2LL * n + i + 1), v[4], y1);
    }
    return make_float2(y0, y1);
}

// Symmetric preconditioner stored by its upper diagonals only: U[d][i] =
// P(i, i+d), d = 0..3 (16 B per row instead of the band's 28 B, so the inner
// iteration's working set stays in L2 to larger n).  The lower entries of
// pair (i, i+1) come from earlier rows, P(i, i-d) = U[d][i-d]; v[k] is window
// row i-4+k.  Out-of-matrix entries multiply window zeros and are not loaded.
__device__ __forceinline__ float2 pair_sym_f(const float *__restrict__ U, int n, int i,
                                             const float (&v)[10]) {
    const float2 z2 = make_float2(0.0f, 0.0f);
    if (!AIRGA_CK(i, 0, n - 1, 604)) return z2;
    const float2 *U0 = reinterpret_cast<const float2 *>(U);
    const float2 *U1 = reinterpret_cast<const float2 *>(U + n);
    const float2 *U2 = reinterpret_cast<const float2 *>(U + 2 * (long long)n);
    const float2 *U3 = reinterpret_cast<const float2 *>(U + 3 * (long long)n);
    const int h = i >> 1;                                   // float2 index of rows (i, i+1)
    const float2 u0 = __ldg(U0 + h), u1 = __ldg(U1 + h), u2 = __ldg(U2 + h), u3 = __ldg(U3 + h);
    const float2 l1 = i >= 2 ? __ldg(U1 + h - 1) : z2;      // U1[i-2], U1[i-1]
    const float2 l2 = i >= 2 ? __ldg(U2 + h - 1) : z2;      // U2[i-2], U2[i-1]
    const float2 l3a = i >= 4 ? __ldg(U3 + h - 2) : z2;     // U3[i-4], U3[i-3]
    const float2 l3b = i >= 2 ? __ldg(U3 + h - 1) : z2;     // U3[i-2], U3[i-1]
    // offsets d = -3 .. 3 in the band kernel's order: for a symmetric band the
    // result is the full-band product bit for bit
    float y0 = l3a.y * v[1];
    y0 = fmaf(l2.x, v[2], y0);
    y0 = fmaf(l1.y, v[3], y0);
    y0 = fmaf(u0.x, v[4], y0);
    y0 = fmaf(u1.x, v[5], y0);
    y0 = fmaf(u2.x, v[6], y0);
    y0 = fmaf(u3.x, v[7], y0);
    float y1 = l3b.x * v[2];
    y1 = fmaf(l2.y, v[3], y1);
    y1 = fmaf(u1.x, v[4], y1);
    y1 = fmaf(u0.y, v[5], y1);
    y1 = fmaf(u1.y, v[6], y1);
    y1 = fmaf(u2.y, v[7], y1);
    y1 = fmaf(u3.y, v[8], y1);
    return make_float2(y0, y1);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-sum NV FP32 values of the inner solve with a shared-memory tree in
// FP32 (the FMA pipe: a handful of cycles per level, where an FP64 level
// occupies a sub-partition's FP64 pipe for 64 cycles); thread 0 of warp q
// writes the CTA's sum of value q, widened to FP64, to partials[slot][q][cta].
// The grid totals and the step lengths stay FP64: summed or divided in FP32
// they cost the inner solve a third more iterations on the precision
// workload.  `red` holds NV * nt floats; blockDim.x must be a multiple of 128.
template <int NV>
__device__ void block_partials_tree_f(float (&v)[NV], float *red, double *partials, int slot,
                                      int grid, int rank) {
    const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * nt + tid] = v[q];
    __syncthreads();
    const int quarter = nt >> 2;
    if (tid < quarter) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            float *r = red + q * nt;
            r[tid] = (r[tid] + r[tid + quarter]) + (r[tid + 2 * quarter] + r[tid + 3 * quarter]);
        }
    }
    __syncthreads();
    const int w = tid >> 5, l = tid & 31;
    if (w < NV) {
        const float *r = red + w * nt;
        float t = 0.0f;
        for (int k = l; k < quarter; k += 32) t += r[k];
        t = warp_sum_f(t);
        if (l == 0) partials[(slot * 4 + w) * grid + rank] = (double)t;
    }
}

template <int MODE>   // 0: identity, 1: band preconditioner, 2: symmetric (upper diagonals)
__global__ void __launch_bounds__(kThreads, 1)
mixed_pair_kernel(Args32 a, int R) {
    extern __shared__ __align__(16) double smem64[];
    __shared__ double tot[8];
    __shared__ int s_flag;
    __shared__ int s_dec;

    const int G = gridDim.x;
    const int n = a.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lo = blockIdx.x * R < n ? blockIdx.x * R : n;
    const int hi = lo + R < n ? lo + R : n;

    double *red = smem64;                                        // 3 * nt doubles
    float *redf = reinterpret_cast<float *>(red);                // the inner loop's FP32 trees
    float *xs = reinterpret_cast<float *>(red + 3 * nt);
    float *rs = xs + R;
    float *ps = rs + (R + 2 * HR);
    float *zq = ps + (R + 2 * HZ);
    float2 *ah = reinterpret_cast<float2 *>(zq + (R + 2 * HZ));  // A rows of the r halo
    const int xbase = lo, rbase = lo - HR, pbase = lo - HZ, zbase = lo - HZ;
    const int lenR = R + 2 * HR, lenZ = R + 2 * HZ;      // window lengths (r; p and z/q)
    (void)lenR;
    (void)lenZ;
    const int rlo = lo - HR > 0 ? lo - HR : 0, rhi = hi + HR < n ? hi + HR : n;
    const int zlo = lo - HZ > 0 ? lo - HZ : 0, zhi = hi + HZ < n ? hi + HZ : n;
    const int bw = HP < (hi - lo) ? HP : (hi - lo);
    const bool packed = a.Apk != nullptr && a.pairz != nullptr && *a.pairz != 0;
    const int hslot = nt - 1 - tid;
    const bool halo_thread = hslot < kHaloPairs;
    const int hpair = hslot < kHaloPairs / 2 ? lo - HR + 2 * hslot : hi + 2 * (hslot - kHaloPairs / 2);
    const bool hvalid = halo_thread && hpair >= 0 && hpair < n;

    {
        const int total = 4 * R + 2 * (HR + 2 * HZ);
        for (int k = tid; k < total; k += nt) xs[k] = 0.0f;
        if (hvalid) {
            float2 t[kBand];
            load_band_pair_f(a.A, n, hpair, t);
#pragma unroll
            for (int d = 0; d < kBand; ++d) ah[hslot * kBand + d] = t[d];
        }
        for (int i = lo + tid; i < hi; i += nt) a.x64[i] = 0.0;   // x_0 = 0
    }
    __syncthreads();

    unsigned bar_no = 0;
    const long long tmo = a.timeout_ns;
    int status = AIRGA_E_MAXIT;
    int inner_total = 0, outer = 0;
    double relres = 0.0;

    // z = M r for the pairs [from, to) (stride 2 nt starting at this thread's
    // slot); r.z and r.r of own pairs accumulate into v2
    auto apply_M = [&](int from, int to, float (&v2)[2]) {
        for (int i = from + 2 * tid; i < to; i += 2 * nt) {
            float2 z;
            if (MODE == 1) {
                float2 pb[kBand];
                load_band_pair_f(a.M, n, i, pb);
                float v[10];
                load_win_f(rs, rbase, i, v, lenR);
                z = pair_full_f(pb, v);
            } else if (MODE == 2) {
                float v[10];
                load_win_f(rs, rbase, i, v, lenR);
                z = pair_sym_f(a.M, n, i, v);
            } else {
                z = AIRGA_CK(i - rbase, 0, lenR - 1, 605)
                        ? *reinterpret_cast<const float2 *>(rs + (i - rbase))
                        : make_float2(0.0f, 0.0f);
            }
            if (AIRGA_CK(i - zbase, 0, lenZ - 1, 606))
                *reinterpret_cast<float2 *>(zq + (i - zbase)) = z;
            if (i >= lo && i < hi) {
                const float2 r = *reinterpret_cast<const float2 *>(rs + (i - rbase));
                v2[0] = fmaf(r.x, z.x, fmaf(r.y, z.y, v2[0]));
                v2[1] = fmaf(r.x, r.x, fmaf(r.y, r.y, v2[1]));
            }
        }
    };

    for (int ko = 0;; ++ko) {
        // ---- FP64 residual r = f - A x on own +- HR into the FP32 window;
        //      ||r||^2 of own rows; x's halo rows were written by the
        //      neighbours before the barrier that ended the previous step ----
        {
            double rr = 0.0;
            for (int i = rlo + tid; i < rhi; i += nt) {
                double r = __ldg(a.f + i);
                if (ko > 0) {
                    double ax = 0.0;
#pragma unroll
                    for (int d = 0; d < kBand; ++d) {
                        const int c = i + d - kHalf;
                        if (c >= 0 && c < n)
                            ax = fma(__ldg(a.A64 + (long long)d * n + i), __ldcg(a.x64 + c), ax);
                    }
                    r -= ax;
                }
                if (AIRGA_CK(i - rbase, 0, lenR, 607)) rs[i - rbase] = (float)r;
                if (i >= lo && i < hi) rr = fma(r, r, rr);
            }
            double v[1] = {rr};
            block_partials_tree<1>(v, red, a.partials, bar_no & 1, G, blockIdx.x);
        }
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
            status = AIRGA_E_TIMEOUT;
            break;
        }
        if (tid < 32) {
            double t[1];
            warp0_totals<1>(a.partials, bar_no & 1, G, t);
            if (tid == 0) {
                const double rr = t[0];
                if (ko == 0) tot[5] = rr;                       // x = 0: r = f
                const double nf2 = tot[5];
                tot[6] = nf2 > 0.0 ? sqrt(rr / nf2) : 0.0;
                s_dec = rr <= a.tol * a.tol * nf2 ? 1 : (ko >= a.max_outer ? 2 : 0);
            }
        }
        __syncthreads();
        ++bar_no;
        relres = tot[6];
        outer = ko;
        if (s_dec == 1) { status = AIRGA_OK; break; }
        if (s_dec == 2) { status = AIRGA_E_MAXIT; break; }

        // ---- FP32 inner PCG: A d = r, d_0 = 0 ----
        for (int i = lo + tid; i < hi; i += nt) xs[i - xbase] = 0.0f;
        int istatus = AIRGA_E_MAXIT;
        int iters = 0;
        {
            float v2[2] = {0.0f, 0.0f};
            apply_M(zlo, zhi, v2);
            block_partials_tree_f<2>(v2, redf, a.partials, bar_no & 1, G, blockIdx.x);
        }
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
            status = AIRGA_E_TIMEOUT;
            break;
        }
        if (tid < 32) {
            double t0[2];
            warp0_totals<2>(a.partials, bar_no & 1, G, t0);
            if (tid == 0) {
                tot[0] = t0[0];                                  // (r, z)
                tot[1] = t0[1];                                  // (r, r)
                s_dec = t0[1] == 0.0 ? 1 : ((!isfinite(t0[0]) || t0[0] == 0.0) ? 2 : 0);
            }
        }
        __syncthreads();
        ++bar_no;
        if (s_dec == 2) istatus = AIRGA_E_BREAKDOWN;
        if (s_dec == 0) {
            double rz = tot[0];
            const double thr2 = a.inner_tol * a.inner_tol * tot[1];
            float beta = 0.0f;
            for (int k = 1; k <= a.maxit; ++k) {
                for (int i = zlo + 2 * tid; i < zhi; i += 2 * nt) {
                    if (!AIRGA_CK(i - pbase, 0, lenZ - 1, 608)) continue;
                    float2 *pp = reinterpret_cast<float2 *>(ps + (i - pbase));
                    const float2 z = *reinterpret_cast<const float2 *>(zq + (i - zbase));
                    if (k == 1) {
                        *pp = z;
                    } else {
                        float2 p = *pp;
                        p.x = fmaf(beta, p.x, z.x);
                        p.y = fmaf(beta, p.y, z.y);
                        *pp = p;
                    }
                }
                __syncthreads();
                for (int t = tid; t < 2 * bw; t += nt) {
                    const int i = t < bw ? lo + t : hi - bw + (t - bw);
                    if (AIRGA_CK(i, 0, n, 609) && AIRGA_CK(i - pbase, 0, lenZ, 609))
                        a.pbuf[i] = ps[i - pbase];
                }
                float vq = 0.0f;
                for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
                    float v[10];
                    load_win_f(ps, pbase, i, v, lenZ);
                    float2 q;
                    if (packed) {
                        q = pair_packed_f(a.Apk, a.A, n, i, v);
                    } else {
                        float2 ab[kBand];
                        load_band_pair_f(a.A, n, i, ab);
                        q = pair_full_f(ab, v);
                    }
                    if (AIRGA_CK(i - zbase, 0, lenZ - 1, 610))
                        *reinterpret_cast<float2 *>(zq + (i - zbase)) = q;
                    vq = fmaf(v[4], q.x, fmaf(v[5], q.y, vq));
                }
                if (MODE != 0 && zlo + 2 * tid < zhi)
                    prefetch_pair_f(a.M, n, zlo + 2 * tid, MODE == 2 ? 4 : kBand);
                {
                    float vv[1] = {vq};
                    block_partials_tree_f<1>(vv, redf, a.partials, bar_no & 1, G, blockIdx.x);
                }
                const bool arrive = !(a.fault_skip_arrival && ko == 0 && k == 1 && blockIdx.x == 0);
                if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag,
                                  arrive)) {
                    istatus = AIRGA_E_TIMEOUT;
                    iters = k - 1;
                    break;
                }
                if (tid < 32) {
                    double pqt[1];
                    warp0_totals<1>(a.partials, bar_no & 1, G, pqt);
                    if (tid == 0) {
                        const double pq = pqt[0];
                        const bool bad = !(pq > 0.0) || !isfinite(pq);
                        s_dec = bad ? 1 : 0;
                        tot[2] = bad ? 0.0 : rz * lean::rcp_signed(pq);
                    }
                }
                __syncthreads();
                ++bar_no;
                if (s_dec) {
                    istatus = AIRGA_E_BREAKDOWN;
                    iters = k - 1;
                    break;
                }
                const float alpha = (float)tot[2];

                float pv[10];
                if (hvalid) {
#pragma unroll
                    for (int q = 0; q < 10; ++q) {
                        const int row = hpair - 4 + q;
                        float v = 0.0f;
                        if (row >= 0 && row < n)
                            v = (row >= lo - HZ && row < hi + HZ) ? ps[row - pbase] : __ldcg(a.pbuf + row);
                        pv[q] = v;
                    }
                }
                for (int i = lo + 2 * tid; i < hi; i += 2 * nt) {
                    if (!AIRGA_CK(i - xbase, 0, R - 1, 611) || !AIRGA_CK(i - rbase, 0, lenR - 1, 611))
                        continue;
                    float2 *xp = reinterpret_cast<float2 *>(xs + (i - xbase));
                    float2 *rp = reinterpret_cast<float2 *>(rs + (i - rbase));
                    const float2 p = *reinterpret_cast<const float2 *>(ps + (i - pbase));
                    const float2 q = *reinterpret_cast<const float2 *>(zq + (i - zbase));
                    float2 x = *xp, r = *rp;
                    x.x = fmaf(alpha, p.x, x.x);
                    x.y = fmaf(alpha, p.y, x.y);
                    r.x = fmaf(-alpha, q.x, r.x);
                    r.y = fmaf(-alpha, q.y, r.y);
                    *xp = x;
                    *rp = r;
                }
                if (hvalid) {
                    float2 t[kBand];
#pragma unroll
                    for (int d = 0; d < kBand; ++d) t[d] = ah[hslot * kBand + d];
                    const float2 q = pair_full_f(t, pv);
                    if (AIRGA_CK(hpair - rbase, 0, lenR - 1, 612)) {
                        float2 *rp = reinterpret_cast<float2 *>(rs + (hpair - rbase));
                        float2 r = *rp;
                        r.x = fmaf(-alpha, q.x, r.x);
                        r.y = fmaf(-alpha, q.y, r.y);
                        *rp = r;
                    }
                }
                __syncthreads();
                float v2[2] = {0.0f, 0.0f};
                apply_M(zlo, zhi, v2);
                if (lo + 2 * tid < hi) {
                    if (packed) prefetch_pair_f(a.Apk, n, lo + 2 * tid, 5);
                    else prefetch_pair_f(a.A, n, lo + 2 * tid, kBand);
                }
                block_partials_tree_f<2>(v2, redf, a.partials, bar_no & 1, G, blockIdx.x);
                if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
                    istatus = AIRGA_E_TIMEOUT;
                    iters = k;
                    break;
                }
                if (tid < 32) {
                    double t2v[2];
                    warp0_totals<2>(a.partials, bar_no & 1, G, t2v);
                    if (tid == 0) {
                        const double rz_new = t2v[0];
                        int dec = 0;
                        if (t2v[1] <= thr2) dec = 1;
                        else if (!isfinite(rz_new) || rz_new == 0.0) dec = 2;
                        s_dec = dec;
                        tot[3] = dec ? 0.0 : rz_new * lean::rcp_signed(rz);
                        tot[4] = rz_new;
                    }
                }
                __syncthreads();
                ++bar_no;
                iters = k;
                {
                    const int dec = s_dec;
                    if (dec == 1) { istatus = AIRGA_OK; break; }
                    if (dec == 2) { istatus = AIRGA_E_BREAKDOWN; break; }
                }
                beta = (float)tot[3];
                rz = tot[4];
            }
        }
        inner_total += iters;
        if (istatus == AIRGA_E_TIMEOUT) { status = istatus; break; }
        // ---- x += d in FP64 (own rows); the barrier publishes x's rows to
        //      the neighbours' next residual.  An inner solve that stopped on
        //      its cap still improved x; a breakdown ends the column. ----
        __syncthreads();
        for (int i = lo + tid; i < hi; i += nt) a.x64[i] += (double)xs[i - xbase];
        if (istatus == AIRGA_E_BREAKDOWN) { status = istatus; outer = ko + 1; break; }
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
            status = AIRGA_E_TIMEOUT;
            break;
        }
        ++bar_no;
    }
    if (blockIdx.x == 0 && tid == 0) {
        *a.relres = relres;
        *a.outer_iters = outer;
        *a.inner_iters = inner_total;
        *a.status = status;
    }
}

size_t mixed_smem(int64_t R) {
    return (size_t)3 * kThreads * sizeof(double) +
           (size_t)(4 * R + 2 * (HR + 2 * HZ) + 2 * kHaloPairs * kBand) * sizeof(float);
}

template <int MODE>
cudaError_t launch_mixed(int grid, int64_t R, size_t smem, const Args32 &args, cudaStream_t s) {
    auto kern = mixed_pair_kernel<MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    Args32 a = args;
    int r = (int)R;
    void *kargs[] = {(void *)&a, (void *)&r};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(kThreads), kargs, smem, s);
}

template <int MODE>
int occupancy_mixed(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(mixed_pair_kernel<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, mixed_pair_kernel<MODE>, kThreads,
                                                          smem);
    return e == cudaSuccess ? AIRGA_OK : cuda_fail(e, "mixed-precision kernel occupancy");
}

int grid_for(int64_t work) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + 255) / 256, cap = (int64_t)sms * 8;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace
}  // namespace airga

using namespace airga;

extern "C" int airga_pcg_solve_mixed(airga_mat A, airga_precond P, const double *F, int32_t m,
                                     const airga_options *opt, double *X, int32_t *outer_iters,
                                     int32_t *inner_iters, int32_t *status, double *true_relres,
                                     void *stream) {
    TraceScope trace_("airga_pcg_solve_mixed", stream);
    int st = check_mat(A, "A");
    if (st) return st;
    if (m < 0) return fail(AIRGA_E_INVALID_ARG, "m must be >= 0");
    if (m == 0) return AIRGA_OK;
    if (!F || !X || !outer_iters || !inner_iters || !status || !true_relres)
        return fail(AIRGA_E_INVALID_ARG, "F, X, outer_iters, inner_iters, status, true_relres are required");
    if (P && (P->n != A->n || P->factors.size() != 1))
        return fail(AIRGA_E_INVALID_ARG, "mixed solve takes no preconditioner or a single-factor one");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    st = check_options(&o);
    if (st) return st;
    const int64_t n = A->n;
    if (n % 2 != 0 || n > (int64_t)INT32_MAX / 8)
        return fail(AIRGA_E_INVALID_ARG, "mixed solve needs an even n below 2^28");
    int dev = 0, sms = 0, optin = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // 2: P_sym stored by its upper diagonals; 1: a nonsymmetric band (symmetrize = 0)
    const int mode = P ? ((o.symmetrize && P->psym) ? 2 : 1) : 0;
    int64_t want = (n + 127) / 128;
    int grid = (int)(want < sms ? want : sms);
    if (grid < 1) grid = 1;
    int64_t R = (n + grid - 1) / grid;
    R += R & 1;
    const size_t smem = mixed_smem(R);
    if (smem + 256 > (size_t)optin)
        return fail(AIRGA_E_INVALID_ARG, "mixed solve: the FP32 state does not fit in shared memory");
    int per_sm = 0;
    st = mode == 2 ? occupancy_mixed<2>(smem, &per_sm)
                   : (mode ? occupancy_mixed<1>(smem, &per_sm) : occupancy_mixed<0>(smem, &per_sm));
    if (st) return st;
    if (per_sm < 1 || grid > per_sm * sms) return fail(AIRGA_E_INVALID_ARG, "mixed solve: grid not co-resident");

    cudaStream_t s = (cudaStream_t)stream;
    // workspace: FP32 A band (7n), FP32 packed (5n), FP32 M band (7n), pbuf32 (n)
    // as floats; partials, control
    const size_t nf = (size_t)n;
    const size_t mfl = mode == 2 ? 4 * nf : (mode ? 7 * nf : 0);
    const size_t floats = 7 * nf + 5 * nf + mfl + nf;
    const size_t doubles = (size_t)8 * grid + 4;
    const size_t bytes = floats * sizeof(float) + 256 + doubles * sizeof(double) + 256;
    void *ws = nullptr;
    st = dev_alloc(&ws, bytes, s);
    if (st) return st;
    char *base = (char *)ws;
    float *A32 = (float *)base;
    float *Apk32 = A32 + 7 * nf;
    float *M32 = Apk32 + 5 * nf;
    float *pbuf = M32 + mfl;
    double *dbase = (double *)(((uintptr_t)(pbuf + nf) + 255) & ~(uintptr_t)255);
    double *partials = dbase;
    unsigned *ctl = (unsigned *)(partials + 8 * grid);

    cudaError_t e = cudaSuccess;
    const int gconv = grid_for(7 * n);
    to_f32_kernel<<<gconv, 256, 0, s>>>(7 * n, A->band->d, A32);
    if (A->pairz) {
        if (!A->packed) {
            st = make_buf(sizeof(double) * 5 * nf, s, &A->packed);
            if (!st) {
                cudaError_t pe = launch_pack_pairs(n, A->band->d, (double *)A->packed.get(), s);
                if (pe != cudaSuccess) st = cuda_fail(pe, "pack pairs");
            }
            if (st) {
                dev_free(ws, s);
                return st;
            }
        }
        to_f32_kernel<<<gconv, 256, 0, s>>>(5 * n, (const double *)A->packed.get(), Apk32);
    }
    if (mode == 2)   // diagonals d = 0..3 of the band are contiguous from row offset 3n
        to_f32_kernel<<<gconv, 256, 0, s>>>(4 * n, P->psym->d + 3 * nf, M32);
    else if (mode)
        to_f32_kernel<<<gconv, 256, 0, s>>>(7 * n, P->factors[0]->d, M32);
    e = cudaGetLastError();
    Args32 a{};
    a.n = (int)n;
    a.A = A32;
    a.Apk = A->pairz ? Apk32 : nullptr;
    a.pairz = A->pairz ? (const int32_t *)A->pairz.get() : nullptr;
    a.M = mode ? M32 : nullptr;
    a.A64 = A->band->d;
    a.pbuf = pbuf;
    a.partials = partials;
    a.bar = ctl;
    a.abort_flag = (int *)(ctl + 1);
    a.tol = o.tol;
    a.inner_tol = o.inner_tol;
    a.maxit = o.maxit;
    a.max_outer = o.max_outer;
    a.timeout_ns = (long long)o.barrier_timeout_ms * 1000000ll;
    const int fault = take_fault(AIRGA_FAULT_SKIP_ARRIVAL) ? 1 : 0;
    // one launch per column runs its whole refinement
    for (int32_t c = 0; c < m && e == cudaSuccess; ++c) {
        a.f = F + (size_t)c * nf;
        a.x64 = X + (size_t)c * nf;
        a.relres = true_relres + c;
        a.outer_iters = outer_iters + c;
        a.inner_iters = inner_iters + c;
        a.status = status + c;
        a.fault_skip_arrival = c == 0 ? fault : 0;
        e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess)
            e = mode == 2 ? launch_mixed<2>(grid, R, smem, a, s)
                          : (mode ? launch_mixed<1>(grid, R, smem, a, s) : launch_mixed<0>(grid, R, smem, a, s));
    }
    dev_free(ws, s);
    if (e != cudaSuccess) return cuda_fail(e, "mixed solve launch");
    return AIRGA_OK;
}

AIRGA_CHECK_READER(mixed)
