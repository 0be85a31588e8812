// Persistent preconditioned CG (one launch per right-hand side column).
//
// The CG recurrence is the standard Hestenes-Stiefel PCG of the paper's CG
// solves (Alg. 3 line 5, Alg. 5 lines 7/11): q = A p; a = (r,z)/(p,q);
// x += a p; r -= a q; z = M r; b = (r,z)_new/(r,z)_old; p = z + b p.
//
// GB300 layout of one iteration
// -----------------------------
// * One cooperative launch of G co-resident CTAs; CTA c owns the rows
//   [lo, hi) = [c R, (c+1) R) for the whole solve.  Two grid barriers per
//   iteration (after (p,q) and after (r,z),(r,r)), each also the only
//   exchange point between CTAs.
// * The vector state of the CTA's rows lives in shared memory when it fits
//   (x: own rows, r: own +- H, p: own +- (H+3), z/q: own +- 3), so per
//   iteration the only DRAM/L2 traffic is the two band-7 matrices A and
//   P_sym (112 B per row) plus a few boundary rows.  When it does not fit,
//   the same windows live in a per-CTA slice of a global workspace.
// * Halo rows are recomputed redundantly instead of exchanged: r on the
//   halo follows r_k = r_{k-1} - a (A p_k) with the same stencil code, and z
//   on own +- 3 from r on own +- H; only p's outer halo is read from the
//   owners (boundary rows written to `pbuf` before barrier 1).  Every CTA
//   therefore holds bit-identical copies of the shared rows.
// * Reductions: warp shuffles -> one partial per CTA -> after the barrier
//   every CTA sums all G partials in the same fixed order, so all CTAs take
//   identical convergence decisions and results are run-to-run deterministic.
// * The barrier is a monotone arrival counter with a bounded wait (global
//   timer); a CTA that gives up sets an abort flag that ends the others'
//   waits, and the column's status becomes AIRGA_E_TIMEOUT.
#include "check.cuh"
#include "pcg_common.cuh"

namespace airga {
namespace {

using namespace pcgdev;

constexpr int kPcgThreads = 512;
constexpr int kMinRowsPerCta = 128;

enum Mode { kIdentity = 0, kBand1 = 1, kChain = 2 };

// One row of (band) x from a window buffer holding rows [wbase, wbase+wlen).
__device__ __forceinline__ double stencil(const double *__restrict__ band, int64_t n, int64_t i,
                                          const double *win, int64_t wbase, int64_t wlen) {
    double acc = 0.0;
    if (!AIRGA_CK(i, 0, n, 201)) return acc;
#pragma unroll
    for (int d = 0; d < kBand; ++d) {
        const int64_t c = i + d - kHalf;
        if (c >= 0 && c < n && AIRGA_CK(c - wbase, 0, wlen, 202))
            acc = fma(__ldg(band + (int64_t)d * n + i), win[c - wbase], acc);
    }
    return acc;
}

// One row of (band)^T x: sum_d F(i+d, i) x_{i+d}, F(i+d, i) = band[(3-d) n + i + d].
__device__ __forceinline__ double stencil_t(const double *__restrict__ band, int64_t n,
                                            int64_t i, const double *win, int64_t wbase,
                                            int64_t wlen) {
    double acc = 0.0;
    if (!AIRGA_CK(i, 0, n, 203)) return acc;
#pragma unroll
    for (int d = -kHalf; d <= kHalf; ++d) {
        const int64_t c = i + d;
        if (c >= 0 && c < n && AIRGA_CK(c - wbase, 0, wlen, 204))
            acc = fma(__ldg(band + (int64_t)(kHalf - d) * n + c), win[c - wbase], acc);
    }
    return acc;
}

// Rows (i, i+1), i even, of (band) x and of (band)^T x from a window whose
// out-of-matrix rows hold zeros (even n, even window base, 16-byte aligned
// band).  Band entries are double2 loads where the pair is aligned (every
// offset of the forward stencil; even offsets of the transposed one) and
// scalar loads otherwise; products are summed in stencil()'s and
// stencil_t()'s order, so each row equals the one-row form (out-of-matrix
// terms are products with window zeros instead of skipped).
__device__ __forceinline__ double2 stencil_pair(const double *__restrict__ band, int64_t n,
                                                int64_t i, const double *win, int64_t wbase,
                                                int64_t wlen) {
    if (!AIRGA_CK(i, 0, n - 1, 205) || !AIRGA_CK(i - 4 - wbase, 0, wlen - 9, 206))
        return make_double2(0.0, 0.0);
    double v[10];
    const double2 *w2 = reinterpret_cast<const double2 *>(win + (i - 4 - wbase));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double2 t = w2[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
    double y0 = 0.0, y1 = 0.0;
#pragma unroll
    for (int d = 0; d < kBand; ++d) {
        const double2 b = __ldg(reinterpret_cast<const double2 *>(band + (int64_t)d * n + i));
        y0 = fma(b.x, v[1 + d], y0);
        y1 = fma(b.y, v[2 + d], y1);
    }
    return make_double2(y0, y1);
}

__device__ __forceinline__ double2 stencil_t_pair(const double *__restrict__ band, int64_t n,
                                                  int64_t i, const double *win, int64_t wbase,
                                                  int64_t wlen) {
    // band reads (3-d) n + i + d .. +1 stay inside the 7 n array for i + 1 < n
    // (entries past a diagonal's ends multiply window zeros)
    if (!AIRGA_CK(i, 0, n - 1, 207) || !AIRGA_CK(i - 4 - wbase, 0, wlen - 9, 208))
        return make_double2(0.0, 0.0);
    double v[10];
    const double2 *w2 = reinterpret_cast<const double2 *>(win + (i - 4 - wbase));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double2 t = w2[k];
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
    double y0 = 0.0, y1 = 0.0;
#pragma unroll
    for (int d = -kHalf; d <= kHalf; ++d) {
        // F(i+d, i) and F(i+1+d, i+1): entries i+d and i+d+1 of band row 3-d
        const double *p = band + (int64_t)(kHalf - d) * n + i + d;
        double b0, b1;
        if ((d & 1) == 0) {
            const double2 b = __ldg(reinterpret_cast<const double2 *>(p));
            b0 = b.x;
            b1 = b.y;
        } else {
            b0 = __ldg(p);
            b1 = __ldg(p + 1);
        }
        y0 = fma(b0, v[4 + d], y0);
        y1 = fma(b1, v[5 + d], y1);
    }
    return make_double2(y0, y1);
}

// z = M r on rows [lo-3, hi+3) (clipped to the matrix), written to zq; the r
// and chain windows hold row i at [i - rbase] (lenR rows each), zq row i at
// [i - lo + 3] (lenZ rows).  PAIRS: the chain stencils run
// by row pairs over each stage's range widened to whole pairs (the extra row
// reads only window rows inside the 2-row pad and feeds no needed row).
template <int MODE, bool PAIRS>
__device__ void apply_precond(const PcgArgs &a, int64_t lo, int64_t hi, int H, int64_t rbase,
                              double *rs, double *zq, double *t1, double *t2, int64_t lenR,
                              int64_t lenZ) {
    (void)lenZ;
    const int64_t n = a.n;
    const int64_t zlo = lo - 3 > 0 ? lo - 3 : 0, zhi = hi + 3 < n ? hi + 3 : n;
    const int64_t zbase = lo - 3;
    if (MODE == kIdentity) {
        for (int64_t i = zlo + threadIdx.x; i < zhi; i += blockDim.x)
            if (AIRGA_CK(i - zbase, 0, lenZ, 209) && AIRGA_CK(i - rbase, 0, lenR, 210))
                zq[i - zbase] = rs[i - rbase];
        return;
    }
    if (MODE == kBand1) {
        const double *Pb = a.psym ? a.psym : a.fac[0];
        for (int64_t i = zlo + threadIdx.x; i < zhi; i += blockDim.x)
            if (AIRGA_CK(i - zbase, 0, lenZ, 211)) zq[i - zbase] = stencil(Pb, n, i, rs, rbase, lenR);
        return;
    }
    // chain: C r with C = F_{nf-1} ... F_0, windows shrink by 3 per factor
    const double *src = rs;
    for (int f = 0; f < a.nf; ++f) {
        const int h = H - 3 * (f + 1);
        const int64_t wlo = lo - h > 0 ? lo - h : 0, whi = hi + h < n ? hi + h : n;
        double *dst = (f & 1) ? t2 : t1;
        if (PAIRS) {
            for (int64_t i = (wlo & ~(int64_t)1) + 2 * threadIdx.x; i < whi; i += 2 * blockDim.x)
                if (AIRGA_CK(i - rbase, 0, lenR - 1, 212))
                    *reinterpret_cast<double2 *>(dst + (i - rbase)) =
                        stencil_pair(a.fac[f], n, i, src, rbase, lenR);
        } else {
            for (int64_t i = wlo + threadIdx.x; i < whi; i += blockDim.x)
                if (AIRGA_CK(i - rbase, 0, lenR, 213))
                    dst[i - rbase] = stencil(a.fac[f], n, i, src, rbase, lenR);
        }
        __syncthreads();
        src = dst;
    }
    if (!a.symmetrize) {
        for (int64_t i = zlo + threadIdx.x; i < zhi; i += blockDim.x)
            if (AIRGA_CK(i - zbase, 0, lenZ, 214) && AIRGA_CK(i - rbase, 0, lenR, 214))
                zq[i - zbase] = src[i - rbase];
        __syncthreads();
        return;
    }
    for (int64_t i = zlo + threadIdx.x; i < zhi; i += blockDim.x)
        if (AIRGA_CK(i - zbase, 0, lenZ, 214) && AIRGA_CK(i - rbase, 0, lenR, 214))
            zq[i - zbase] = src[i - rbase];
    __syncthreads();
    // C^T r = F_0^T ... F_{nf-1}^T r
    src = rs;
    for (int s = 0; s < a.nf; ++s) {
        const int f = a.nf - 1 - s;
        const int h = H - 3 * (s + 1);
        const int64_t wlo = lo - h > 0 ? lo - h : 0, whi = hi + h < n ? hi + h : n;
        double *dst = (s & 1) ? t2 : t1;
        if (PAIRS) {
            for (int64_t i = (wlo & ~(int64_t)1) + 2 * threadIdx.x; i < whi; i += 2 * blockDim.x)
                if (AIRGA_CK(i - rbase, 0, lenR - 1, 215))
                    *reinterpret_cast<double2 *>(dst + (i - rbase)) =
                        stencil_t_pair(a.fac[f], n, i, src, rbase, lenR);
        } else {
            for (int64_t i = wlo + threadIdx.x; i < whi; i += blockDim.x)
                if (AIRGA_CK(i - rbase, 0, lenR, 216))
                    dst[i - rbase] = stencil_t(a.fac[f], n, i, src, rbase, lenR);
        }
        __syncthreads();
        src = dst;
    }
    for (int64_t i = zlo + threadIdx.x; i < zhi; i += blockDim.x)
        if (AIRGA_CK(i - zbase, 0, lenZ, 217) && AIRGA_CK(i - rbase, 0, lenR, 217))
            zq[i - zbase] = 0.5 * (zq[i - zbase] + src[i - rbase]);
}

// SMEM: 0 every window in this CTA's slice of the global workspace; 1 every
// window in shared memory; 2 (update chains) the windows the chain stencils
// read and write — r, t1, t2 — in shared memory, x, p and z/q in the global
// slice (the six windows of a chain do not fit shared memory at large n).
template <int SMEM, int MODE>
__global__ void __launch_bounds__(kPcgThreads, 1)
pcg_kernel(PcgArgs a, int64_t R, int H) {
    extern __shared__ double smem[];
    __shared__ double red[160];
    __shared__ int s_flag;

    const int G = gridDim.x;
    const int64_t n = a.n;
    const int64_t lo = (int64_t)blockIdx.x * R < n ? (int64_t)blockIdx.x * R : n;
    const int64_t hi = lo + R < n ? lo + R : n;
    const int tid = threadIdx.x, nt = blockDim.x;

    // window buffers (global row i of a window with base B sits at buf[i - B])
    // chain windows in shared memory (SMEM == 2) run row-pair stencils: even
    // base and a 2-row pad on each side, zeroed once (rows outside the
    // matrix must read as zeros)
    constexpr int64_t kPad = SMEM == 2 ? 2 : 0;
    const int64_t lenX = R, lenR = R + 2 * H + 2 * kPad, lenP = R + 2 * H + 6, lenZ = R + 6;
    double *xs, *rs, *ps, *zq, *t1 = nullptr, *t2 = nullptr;
    if (SMEM == 2) {
        rs = smem;
        t1 = rs + lenR;
        t2 = t1 + lenR;
        xs = a.state + (size_t)blockIdx.x * (lenX + lenP + lenZ);
        ps = xs + lenX;
        zq = ps + lenP;
    } else {
        double *base = SMEM ? smem : a.state + (size_t)blockIdx.x * (lenX + lenR + lenP + lenZ + 2 * lenR);
        xs = base;
        rs = xs + lenX;
        ps = rs + lenR;
        zq = ps + lenP;
        if (!SMEM) {
            t1 = zq + lenZ;
            t2 = t1 + lenR;
        }
    }
    const int64_t xbase = lo, rbase = lo - H - kPad, pbase = lo - H - 3, zbase = lo - 3;
    const int64_t rlo = lo - H > 0 ? lo - H : 0, rhi = hi + H < n ? hi + H : n;
    const int64_t plo3 = lo - 3 > 0 ? lo - 3 : 0, phi3 = hi + 3 < n ? hi + 3 : n;
    const int64_t bw = (H + 3) < (hi - lo) ? (H + 3) : (hi - lo);   // boundary rows written

    unsigned bar_no = 0;
    const long long tmo = a.timeout_ns;
    int status = AIRGA_E_MAXIT;
    int iters = 0;

    if (SMEM == 2) {
        for (int64_t k = tid; k < 3 * lenR; k += nt) smem[k] = 0.0;
        __syncthreads();
    }
    // ---- initial residual r_0 = b - A x_0 on own +- H, x_0 on own rows ----
    for (int64_t i = lo + tid; i < hi; i += nt) xs[i - xbase] = a.warm ? a.x[i] : 0.0;
    for (int64_t i = rlo + tid; i < rhi; i += nt) {
        double v = a.b[i];
        if (a.warm) {
            double ax = 0.0;
#pragma unroll
            for (int d = 0; d < kBand; ++d) {
                const int64_t c = i + d - kHalf;
                if (c >= 0 && c < n) ax = fma(__ldg(a.A + (int64_t)d * n + i), a.x[c], ax);
            }
            v -= ax;
        }
        if (AIRGA_CK(i - rbase, 0, lenR, 218)) rs[i - rbase] = v;
    }
    __syncthreads();
    apply_precond<MODE, SMEM == 2>(a, lo, hi, H, rbase, rs, zq, t1, t2, lenR, lenZ);
    __syncthreads();
    {
        double v[3] = {0.0, 0.0, 0.0};
        for (int64_t i = lo + tid; i < hi; i += nt) {
            const double r = rs[i - rbase], bi = a.b[i];
            v[0] = fma(r, zq[i - zbase], v[0]);
            v[1] = fma(r, r, v[1]);
            v[2] = fma(bi, bi, v[2]);
        }
        block_partials<3>(v, red, a.partials, bar_no & 1, G);
    }
    if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
        status = AIRGA_E_TIMEOUT;
        goto finish;
    }
    double tot0[3];
    grid_totals<3>(a.partials, bar_no & 1, G, red + 128, tot0);
    ++bar_no;
    {
        double rz = tot0[0];
        const double nb = sqrt(tot0[2]);
        double rn = sqrt(tot0[1]);
        if (blockIdx.x == 0 && tid == 0 && a.hist) a.hist[0] = nb > 0.0 ? rn / nb : 0.0;
        if (nb == 0.0) {
            for (int64_t i = lo + tid; i < hi; i += nt) xs[i - xbase] = 0.0;
            status = AIRGA_OK;
            goto finish;
        }
        if (rn <= a.tol * nb) { status = AIRGA_OK; goto finish; }
        if (!isfinite(rz) || rz == 0.0) { status = AIRGA_E_BREAKDOWN; goto finish; }

        double beta = 0.0;
        for (int k = 1; k <= a.maxit; ++k) {
            // ---- phase 1: p = z + beta p on own +- 3; boundary rows out; q = A p ----
            if (k == 1) {
                for (int64_t i = plo3 + tid; i < phi3; i += nt)
                    if (AIRGA_CK(i - pbase, 0, lenP, 219) && AIRGA_CK(i - zbase, 0, lenZ, 219))
                        ps[i - pbase] = zq[i - zbase];
            } else {
                for (int64_t i = plo3 + tid; i < phi3; i += nt)
                    if (AIRGA_CK(i - pbase, 0, lenP, 219) && AIRGA_CK(i - zbase, 0, lenZ, 219))
                        ps[i - pbase] = fma(beta, ps[i - pbase], zq[i - zbase]);
            }
            __syncthreads();
            for (int64_t t = tid; t < 2 * bw; t += nt) {
                const int64_t i = t < bw ? lo + t : hi - bw + (t - bw);
                if (AIRGA_CK(i, 0, n, 220) && AIRGA_CK(i - pbase, 0, lenP, 220))
                    a.pbuf[i] = ps[i - pbase];
            }
            double vq[1] = {0.0};
            for (int64_t i = lo + tid; i < hi; i += nt) {
                const double q = stencil(a.A, n, i, ps, pbase, lenP);
                if (AIRGA_CK(i - zbase, 0, lenZ, 221)) zq[i - zbase] = q;
                vq[0] = fma(ps[i - pbase], q, vq[0]);
            }
            block_partials<1>(vq, red, a.partials, bar_no & 1, G);
            const bool arrive = !(a.fault_skip_arrival && k == 1 && blockIdx.x == 0);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag,
                              arrive)) {
                status = AIRGA_E_TIMEOUT;
                iters = k - 1;
                goto finish;
            }
            double pqt[1];
            grid_totals<1>(a.partials, bar_no & 1, G, red + 128, pqt);
            ++bar_no;
            const double pq = pqt[0];
            if (!(pq > 0.0) || !isfinite(pq)) {
                status = AIRGA_E_BREAKDOWN;
                iters = k - 1;
                goto finish;
            }
            const double alpha = rz / pq;

            // ---- phase 2: outer p halo in; x, r updates; z = M r ----
            for (int64_t t = tid; t < 2 * (int64_t)H; t += nt) {
                const int64_t i = t < H ? lo - H - 3 + t : hi + 3 + (t - H);
                if (i < 0 || i >= n || !AIRGA_CK(i - pbase, 0, lenP, 222)) continue;
                ps[i - pbase] = __ldcg(a.pbuf + i);
            }
            for (int64_t i = lo + tid; i < hi; i += nt) {
                if (!AIRGA_CK(i - xbase, 0, lenX, 223)) continue;
                xs[i - xbase] = fma(alpha, ps[i - pbase], xs[i - xbase]);
                rs[i - rbase] = fma(-alpha, zq[i - zbase], rs[i - rbase]);
            }
            __syncthreads();
            for (int64_t t = tid; t < 2 * (int64_t)H; t += nt) {
                const int64_t i = t < H ? lo - H + t : hi + (t - H);
                if (i < 0 || i >= n || !AIRGA_CK(i - rbase, 0, lenR, 224)) continue;
                rs[i - rbase] = fma(-alpha, stencil(a.A, n, i, ps, pbase, lenP), rs[i - rbase]);
            }
            __syncthreads();
            apply_precond<MODE, SMEM == 2>(a, lo, hi, H, rbase, rs, zq, t1, t2, lenR, lenZ);
            __syncthreads();
            double v2[2] = {0.0, 0.0};
            for (int64_t i = lo + tid; i < hi; i += nt) {
                const double r = rs[i - rbase];
                v2[0] = fma(r, zq[i - zbase], v2[0]);
                v2[1] = fma(r, r, v2[1]);
            }
            block_partials<2>(v2, red, a.partials, bar_no & 1, G);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
                status = AIRGA_E_TIMEOUT;
                iters = k;
                goto finish;
            }
            double t2v[2];
            grid_totals<2>(a.partials, bar_no & 1, G, red + 128, t2v);
            ++bar_no;
            iters = k;
            rn = sqrt(t2v[1]);
            if (blockIdx.x == 0 && tid == 0 && a.hist) a.hist[k] = rn / nb;
            if (rn <= a.tol * nb) { status = AIRGA_OK; break; }
            const double rz_new = t2v[0];
            if (!isfinite(rz_new) || rz_new == 0.0) { status = AIRGA_E_BREAKDOWN; break; }
            beta = rz_new / rz;
            rz = rz_new;
        }
    }
finish:
    __syncthreads();
    for (int64_t i = lo + tid; i < hi; i += nt) a.x[i] = xs[i - xbase];
    if (blockIdx.x == 0 && tid == 0) {
        *a.iters = iters;
        *a.status = status;
    }
}

template <int SMEM, int MODE>
cudaError_t launch_mode(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s) {
    auto kern = pcg_kernel<SMEM, MODE>;
    if (SMEM) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan.smem_bytes);
        if (e != cudaSuccess) return e;
    }
    PcgArgs a = args;
    int64_t R = plan.rows;
    int H = plan.halo;
    void *kargs[] = {(void *)&a, (void *)&R, (void *)&H};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(plan.grid), dim3(plan.threads),
                                       kargs, SMEM ? plan.smem_bytes : 0, s);
}

int mode_of(int nf, bool psym_path) {
    if (nf == 0) return kIdentity;
    if (nf == 1) return kBand1;
    (void)psym_path;
    return kChain;
}

}  // namespace

int pcg_plan(int64_t n, int nf, bool psym_path, bool aligned16, int device, PcgPlan *plan,
             int share) {
    const int mode = mode_of(nf, psym_path);
    int sms = 0, optin = 0, smem_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    const int forced = forced_pcg_kind();
    // node-pair kernel: even n, aligned operands, no update chain; state in
    // shared memory (kind 2), or r and p in shared memory with x and z/q in
    // global memory (kind 3).  Automatic order 2, 3, generic; a forced kind is
    // taken first when it applies.
    if (mode != kChain && aligned16 && n % 2 == 0 && forced != 1) {
        int64_t want_p = (n + kMinRowsPerCta - 1) / kMinRowsPerCta;
        int grid_p = (int)(want_p < sms ? want_p : sms);
        if (grid_p < 1) grid_p = 1;
        int64_t Rp = (n + grid_p - 1) / grid_p;
        Rp += Rp & 1;
        const size_t smem_p = pcg_pair_smem(Rp), smem_s = pcg_pair_split_smem(Rp);
        bool ok2 = false, ok3 = false, ok4 = false;
        if (share == 2 || share == 3 || forced == 4) {
            // half an SM: one CTA of each of two solves per SM.  Footprint of a
            // CTA = dynamic + static shared memory + the per-block reservation.
            // A lead (share 2) pads its dynamic request so that its footprint is
            // just over half the SM: two lead CTAs never share an SM, so the
            // dispatcher has to spread a lead one CTA per SM even when other
            // work holds some SMs at its launch (a doubled-up SM would pace the
            // whole solve).  A partner (share 3, or the test hook) must fit in
            // the rest of every SM.
            const int md = mode == kIdentity ? 0 : 1;
            const size_t smem_h = pcg_pair_half_smem(Rp);
            int reserved = 0;
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
            const size_t stat = pcg_pair_half_static_smem(md) + (size_t)reserved;
            const size_t half_sm = (size_t)smem_sm / 2;
            const size_t lead = half_sm + 64 > stat ? half_sm + 64 - stat : smem_h;
            size_t smem_use = smem_h;
            if (smem_h + stat + 64 <= half_sm && lead + 256 <= (size_t)optin) {
                int per_sm = 0;
                if (share == 2) {
                    int st = pcg_pair_half_occupancy(md, lead, &per_sm);
                    if (st) return st;
                    ok4 = per_sm == 1 && grid_p <= sms;
                    smem_use = lead;
                } else {
                    int st = pcg_pair_half_occupancy(md, smem_h, &per_sm);
                    if (st) return st;
                    ok4 = per_sm >= 2 && grid_p <= sms;
                }
            }
            if (ok4) {
                plan->kind = 4;
                plan->threads = pcg_pair_threads(4);
                plan->halo = 8;
                plan->grid = grid_p;
                plan->rows = Rp;
                plan->smem_state = false;
                plan->smem_bytes = smem_use;
                plan->scratch_doubles = pcg_pair_split_slice(Rp) * (size_t)grid_p;
                return AIRGA_OK;
            }
        }
        if (smem_p + 256 <= (size_t)optin) {
            int per_sm = 0;
            int st = pcg_pair_occupancy(mode == kIdentity ? 0 : 1, smem_p, &per_sm);
            if (st) return st;
            ok2 = per_sm >= 1 && grid_p <= per_sm * sms;
        }
        if (smem_s + 256 <= (size_t)optin) {
            int per_sm = 0;
            int st = pcg_pair_split_occupancy(mode == kIdentity ? 0 : 1, smem_s, &per_sm);
            if (st) return st;
            ok3 = per_sm >= 1 && grid_p <= per_sm * sms;
        }
        const int kind = (forced == 3 && ok3) ? 3 : (ok2 ? 2 : (ok3 ? 3 : 0));
        if (kind) {
            plan->kind = kind;
            plan->threads = pcg_pair_threads(kind);
            plan->halo = 8;
            plan->grid = grid_p;
            plan->rows = Rp;
            plan->smem_state = kind == 2;
            plan->smem_bytes = kind == 2 ? smem_p : smem_s;
            plan->scratch_doubles = kind == 2 ? 0 : pcg_pair_split_slice(Rp) * (size_t)grid_p;
            return AIRGA_OK;
        }
    }
    int H = mode == kIdentity ? 3 : (mode == kBand1 ? 6 : 3 + 3 * nf);
    // update chains with even n and aligned operands run their stencils by row
    // pairs in shared memory: even halo and even rows per CTA keep pairs aligned
    const bool chain_pairs = mode == kChain && n % 2 == 0 && aligned16;
    if (chain_pairs) H += H & 1;
    const size_t static_smem = 160 * sizeof(double) + 64;
    // grid: one CTA per SM at most (the state fills shared memory), fewer for
    // small n so that every CTA keeps at least kMinRowsPerCta rows
    int64_t want = (n + kMinRowsPerCta - 1) / kMinRowsPerCta;
    int grid = (int)(want < sms ? want : sms);
    if (grid < 1) grid = 1;
    int64_t R = (n + grid - 1) / grid;
    if (chain_pairs) R += R & 1;
    // shared memory: all four windows (identity, one band), or for a chain the
    // r, t1, t2 windows (2-row pads) with x, p, z/q in a global slice
    const size_t per_cta = mode == kChain ? (size_t)3 * (R + 2 * H + 4)
                                          : (size_t)(R + (R + 2 * H) + (R + 2 * H + 6) + (R + 6));
    const size_t smem = per_cta * sizeof(double);
    plan->threads = kPcgThreads;
    plan->halo = H;
    plan->grid = grid;
    plan->rows = R;
    plan->smem_state = (smem + static_smem <= (size_t)optin) && forced != 1 &&
                       (mode != kChain || chain_pairs);
    plan->kind = plan->smem_state ? 0 : 1;
    plan->smem_bytes = plan->smem_state ? smem : 0;
    const size_t slice = (size_t)(R + (R + 2 * H) + (R + 2 * H + 6) + (R + 6) + 2 * (R + 2 * H));
    const size_t chain_slice = (size_t)(R + (R + 2 * H + 6) + (R + 6));
    plan->scratch_doubles = !plan->smem_state ? slice * (size_t)grid
                            : (mode == kChain ? chain_slice * (size_t)grid : 0);
    // co-residency check for the cooperative launch
    int per_sm = 0;
    cudaError_t e;
    if (plan->smem_state) {
        const void *kern = mode == kIdentity ? (const void *)pcg_kernel<1, kIdentity>
                         : mode == kBand1    ? (const void *)pcg_kernel<1, kBand1>
                                             : (const void *)pcg_kernel<2, kChain>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail(AIRGA_E_CUDA, "pcg: cannot reserve shared memory");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPcgThreads, smem);
    } else {
        if (mode == kIdentity)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<0, kIdentity>,
                                                              kPcgThreads, 0);
        else if (mode == kBand1)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<0, kBand1>,
                                                              kPcgThreads, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel<0, kChain>,
                                                              kPcgThreads, 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pcg occupancy");
    if (per_sm < 1 || grid > per_sm * sms)
        return fail(AIRGA_E_INVALID_ARG, "pcg: grid cannot be co-resident");
    return AIRGA_OK;
}

cudaError_t launch_pcg(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s) {
    const cudaError_t fe = injected_launch_error();   // host-side test fault only
    if (fe != cudaSuccess) return fe;
    if (plan.kind >= 2) return launch_pcg_pair(plan, args, s);       // node-pair kinds 2, 3, 4
    const int mode = mode_of(args.nf, args.psym != nullptr);
    if (plan.smem_state) {
        if (mode == kIdentity) return launch_mode<1, kIdentity>(plan, args, s);
        if (mode == kBand1) return launch_mode<1, kBand1>(plan, args, s);
        return launch_mode<2, kChain>(plan, args, s);
    }
    if (mode == kIdentity) return launch_mode<0, kIdentity>(plan, args, s);
    if (mode == kBand1) return launch_mode<0, kBand1>(plan, args, s);
    return launch_mode<0, kChain>(plan, args, s);
}

}  // namespace airga

AIRGA_CHECK_READER(pcg_kernel)
