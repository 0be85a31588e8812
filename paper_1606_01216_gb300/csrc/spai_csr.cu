// SPAI and SPAI update on a general sparsity pattern (Sec. 3.1, Eq. 3.1;
// Sec. 3.2, Algorithms 2 and 4), for matrices kept in CSR storage.
//
// Column j of the preconditioner solves min ||b_j - A m||_2 over vectors m
// supported on J_j (column j of the pattern S): b_j = e_j for a build,
// b_j = A_old e_j for an update.  Only the rows I_j touched by A's columns in
// J_j can change the residual, so the problem is the dense |I_j| x |J_j|
// block A(I_j, J_j).
//
// Two phases:
// * symbolic (once per pair of patterns A, S, cached on A's pattern): I_j of
//   every column as a sorted row list, one warp per column — the rows of the
//   |J_j| columns are gathered into shared memory and each lane keeps the
//   first occurrence of a value and its rank among distinct values;
// * numeric (every build / update): one warp per column, the block in
//   shared memory with lane l holding rows l and l + 32; Householder QR with
//   warp reductions (the textbook triangularisation: reflector
//   v = x + sign(x_1) ||x|| e_1, applied to the trailing columns and to b,
//   then back substitution), or the paper's MR iteration on the same block.
#include "csr_common.cuh"

namespace airga {
namespace {

constexpr int kCand = 512;        // gathered row indices per column (symbolic phase)
constexpr int kRowsWarps = 8;     // warps per CTA in the symbolic kernel
constexpr int kNumWarps = 4;      // warps per CTA in the numeric kernel

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int wsum_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// position of `row` in the sorted list I[0..ni), or -1
__device__ __forceinline__ int find_row(const int32_t *I, int ni, int32_t row) {
    int lo = 0, hi = ni;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (I[mid] < row) lo = mid + 1;
        else hi = mid;
    }
    return (lo < ni && I[lo] == row) ? lo : -1;
}

// ---------------------------------------------------------------------------
// symbolic phase
// ---------------------------------------------------------------------------

// FILL == false: cnt[j + 1] = |I_j|; stats: [0] max |I_j|, [1] max |J_j|,
// [2] error bits (1: |J_j| > kSpaiMaxJ, 2: more than kCand gathered rows,
// 4: |I_j| > kSpaiMaxI).  FILL == true: irows[iptr[j] ..] = I_j, sorted.
template <bool FILL>
__global__ void __launch_bounds__(32 * kRowsWarps)
spai_rows_kernel(int64_t n, const int64_t *__restrict__ Acp, const int32_t *__restrict__ Ari,
                 const int64_t *__restrict__ Scp, const int32_t *__restrict__ Sri,
                 int64_t *__restrict__ cnt, const int64_t *__restrict__ iptr,
                 int32_t *__restrict__ irows, int32_t *stats) {
    __shared__ int32_t cand_all[kRowsWarps][kCand];
    __shared__ unsigned char first_all[kRowsWarps][kCand];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    int32_t *cand = cand_all[wi];
    unsigned char *first = first_all[wi];
    const int64_t nwarps = (int64_t)gridDim.x * kRowsWarps;
    int my_max_i = 0, my_max_j = 0, bits = 0;
    for (int64_t j = blockIdx.x * (int64_t)kRowsWarps + wi; j < n; j += nwarps) {
        const int64_t sb = Scp[j];
        const int nj = (int)(Scp[j + 1] - sb);
        my_max_j = max(my_max_j, nj);
        if (nj > kSpaiMaxJ) {
            bits |= 1;
            if (!FILL) cnt[j + 1] = 0;
            continue;
        }
        // lane c < nj gathers column J_c of A; offsets by a warp scan
        int k = 0, len = 0;
        if (lane < nj) {
            k = Sri[sb + lane];
            len = (int)(Acp[k + 1] - Acp[k]);
        }
        int off = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += y;
        }
        const int m = __shfl_sync(0xffffffffu, off, 31);
        off -= len;
        if (m > kCand) {
            bits |= 2;
            if (!FILL) cnt[j + 1] = 0;
            continue;
        }
        if (lane < nj)
            for (int q = 0; q < len; ++q) cand[off + q] = Ari[Acp[k] + q];
        __syncwarp();
        // first occurrences, then ranks among the distinct values
        for (int t = lane; t < m; t += 32) {
            const int32_t v = cand[t];
            bool f = true;
            for (int u = 0; u < t && f; ++u) f = cand[u] != v;
            first[t] = f ? 1 : 0;
        }
        __syncwarp();
        int distinct = 0;
        for (int t = lane; t < m; t += 32) {
            if (!first[t]) continue;
            ++distinct;
            if (FILL) {
                const int32_t v = cand[t];
                int rank = 0;
                for (int u = 0; u < m; ++u) rank += (first[u] && cand[u] < v) ? 1 : 0;
                irows[iptr[j] + rank] = v;
            }
        }
        distinct = wsum_i(distinct);
        my_max_i = max(my_max_i, distinct);
        if (distinct > kSpaiMaxI) bits |= 4;
        if (!FILL && lane == 0) cnt[j + 1] = distinct;
        __syncwarp();
    }
    if (!FILL && lane == 0) {
        atomicMax(stats, my_max_i);
        atomicMax(stats + 1, my_max_j);
        if (bits) atomicOr(stats + 2, bits);
    }
}

__global__ void __launch_bounds__(1024) scan_kernel(int64_t *a, int64_t len) {
    // one CTA, sequential tiles (the symbolic phase runs once per pattern pair)
    __shared__ int64_t wsum_s[32];
    __shared__ int64_t carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 1024) {
        const int64_t idx = base + tid;
        int64_t v = idx < len ? a[idx] : 0, x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum_s[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = wsum_s[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum_s[lane] = s;
        }
        __syncthreads();
        if (idx < len) a[idx] = carry + (w > 0 ? wsum_s[w - 1] : 0) + x;
        __syncthreads();
        if (tid == 0) carry += wsum_s[31];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// numeric phase
// ---------------------------------------------------------------------------

struct SpaiCsrArgs {
    int64_t n;
    int64_t nnz_a, nnz_s;   // entries of A and of S (bounds of checked builds)
    // A by columns: entries of column k are [Acp[k], Acp[k+1]) with rows Ari
    // and values Av[Atp[e]] (A_old: Aold[Atp[e]], same pattern)
    const int64_t *Acp;
    const int32_t *Ari;
    const int64_t *Atp;
    const double *Av;
    const double *Aold;
    // S by columns and the CSR position of each of its entries
    const int64_t *Scp;
    const int32_t *Sri;
    const int64_t *Stp;
    const int64_t *iptr;
    const int32_t *irows;
    int mr;
    const double *alpha0;
    double tol;
    int relative;
    int kmax;
    double *F;
    int32_t *steps;
    double *colres;
    int32_t *flag;
};

// Shared memory of one warp for R rows per lane: the block Ah (column c at
// Ah + c * 32R), b, the solution / MR iterate, the MR direction and the
// index lists.
template <int R>
struct WarpMem {
    static constexpr int kLd = 32 * R;
    __host__ __device__ static size_t bytes(int max_j) {
        return sizeof(double) * ((size_t)max_j * kLd + kLd + 2 * kSpaiMaxJ) +
               sizeof(int32_t) * (kLd + 2 * kSpaiMaxJ) + sizeof(double) * kSpaiMaxJ;
    }
};

template <int R>
__global__ void __launch_bounds__(32 * kNumWarps)
spai_csr_kernel(SpaiCsrArgs a, int max_j) {
    extern __shared__ __align__(16) double smem_d[];
    constexpr int kLd = WarpMem<R>::kLd;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    char *wbase = reinterpret_cast<char *>(smem_d) + (size_t)wi * WarpMem<R>::bytes(max_j);
    double *Ah = reinterpret_cast<double *>(wbase);
    double *bv = Ah + (size_t)max_j * kLd;
    double *xs = bv + kLd;                       // solution / MR iterate m
    double *dv = xs + kSpaiMaxJ;                 // MR direction; QR: 1 / R_kk
    double *bout = dv + kSpaiMaxJ;               // b at rows J_c outside I_j
    int32_t *Irow = reinterpret_cast<int32_t *>(bout + kSpaiMaxJ);
    int32_t *Jcol = Irow + kLd;
    int32_t *Jpos = Jcol + kSpaiMaxJ;            // position of row J_c in I_j, or -1

    const int64_t nwarps = (int64_t)gridDim.x * kNumWarps;
    for (int64_t j = blockIdx.x * (int64_t)kNumWarps + wi; j < a.n; j += nwarps) {
        const int64_t sb = a.Scp[j];
        const int nj = (int)(a.Scp[j + 1] - sb);
        const int64_t ib = a.iptr[j];
        const int ni = (int)(a.iptr[j + 1] - ib);
        if (!AIRGA_CK(nj, 0, max_j + 1, 401) || !AIRGA_CK(ni, 0, kLd + 1, 402)) continue;
        if (lane < nj) {
            const int32_t c = a.Sri[sb + lane];
            Jcol[lane] = AIRGA_CK(c, 0, a.n, 403) ? c : 0;
        }
        for (int r = lane; r < kLd; r += 32) Irow[r] = r < ni ? a.irows[ib + r] : INT32_MAX;
        for (int c = 0; c < nj; ++c)
            for (int r = lane; r < kLd; r += 32) Ah[c * kLd + r] = 0.0;
        for (int r = lane; r < kLd; r += 32) bv[r] = 0.0;
        __syncwarp();
        // block A(I_j, J_j)
        for (int c = 0; c < nj; ++c) {
            const int64_t k = Jcol[c];
            for (int64_t e = a.Acp[k] + lane; e < a.Acp[k + 1]; e += 32) {
                if (!AIRGA_CK(e, 0, a.nnz_a, 404)) break;
                const int p = find_row(Irow, ni, a.Ari[e]);
                const int64_t t = a.Atp[e];
                if (p >= 0 && AIRGA_CK(t, 0, a.nnz_a, 405)) Ah[c * kLd + p] = a.Av[t];
            }
        }
        // right-hand side on I_j; ||b||^2 outside I_j
        double bo2 = 0.0;
        if (a.Aold) {
            for (int64_t e = a.Acp[j] + lane; e < a.Acp[j + 1]; e += 32) {
                if (!AIRGA_CK(e, 0, a.nnz_a, 406) || !AIRGA_CK(a.Atp[e], 0, a.nnz_a, 406)) break;
                const double v = a.Aold[a.Atp[e]];
                const int p = find_row(Irow, ni, a.Ari[e]);
                if (p >= 0) bv[p] = v;
                else bo2 = fma(v, v, bo2);
            }
            bo2 = wsum(bo2);
        } else if (lane == 0) {
            const int p = find_row(Irow, ni, (int32_t)j);
            if (p >= 0) bv[p] = 1.0;
            else bo2 = 1.0;
        }
        bo2 = __shfl_sync(0xffffffffu, bo2, 0);
        __syncwarp();

        if (!a.mr) {
            // ---------------- Householder QR of the ni x nj block ----------------
            bool rank_bad = ni < nj;
            if (!rank_bad) {
                for (int k = 0; k < nj; ++k) {
                    double *ak = Ah + k * kLd;
                    double x[R];
                    double nx2 = 0.0;
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int r = lane + 32 * q;
                        x[q] = (r >= k && r < ni) ? ak[r] : 0.0;
                        nx2 = fma(x[q], x[q], nx2);
                    }
                    nx2 = wsum(nx2);
                    const double nx = sqrt(nx2);
                    const double xk = ak[k];
                    const double sg = xk >= 0.0 ? 1.0 : -1.0;
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int r = lane + 32 * q;
                        if (r == k) x[q] += sg * nx;     // x now holds v
                    }
                    // ||v||^2 = ||x||^2 - x_k^2 + (x_k + sg ||x||)^2 = 2 ||x|| (||x|| + |x_k|):
                    // no second warp reduction.  Each warp-wide FP64 instruction holds a
                    // sub-partition's FP64 pipe for ~64 cycles whatever the active lanes,
                    // so the reductions and divisions, not the FMAs, set this kernel's
                    // time: one reciprocal per reflector instead of a division per column.
                    const double vv = 2.0 * nx * (nx + fabs(xk));
                    if (vv == 0.0) continue;             // zero column: R_kk = 0, caught below
                    const double tau = 2.0 / vv;
                    for (int t = k; t <= nj; ++t) {      // t == nj: the right-hand side
                        double *col = t < nj ? Ah + t * kLd : bv;
                        double sdot = 0.0;
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            const int r = lane + 32 * q;
                            if (r >= k && r < ni) sdot = fma(x[q], col[r], sdot);
                        }
                        sdot = wsum(sdot) * tau;
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            const int r = lane + 32 * q;
                            if (r >= k && r < ni) col[r] = fma(-sdot, x[q], col[r]);
                        }
                    }
                    __syncwarp();
                }
                double rmax = 0.0;
                for (int k = 0; k < nj; ++k) rmax = fmax(rmax, fabs(Ah[k * kLd + k]));
                for (int k = 0; k < nj; ++k) {
                    const double rkk = Ah[k * kLd + k];
                    if (rkk == 0.0 || fabs(rkk) < 1e-14 * rmax) rank_bad = true;
                }
            }
            if (rank_bad) {
                if (lane == 0) atomicOr(a.flag, 1);
                if (lane < nj) xs[lane] = 0.0;
            } else {
                // the reciprocals of R's diagonal in one warp-wide division (lane k
                // takes R_kk), then the back substitution R x = (Q^T b)(0:nj) by lane 0
                if (lane < nj) dv[lane] = 1.0 / Ah[lane * kLd + lane];
                __syncwarp();
                if (lane == 0) {
                    for (int k = nj - 1; k >= 0; --k) {
                        double s = bv[k];
                        for (int t = k + 1; t < nj; ++t) s = fma(-Ah[t * kLd + k], xs[t], s);
                        xs[k] = s * dv[k];
                    }
                }
            }
            __syncwarp();
            if (a.colres) {
                // ||b - A m||^2 = ||(Q^T b)(nj:ni)||^2 + the part of b outside I_j
                double rr = 0.0;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int r = lane + 32 * q;
                    if (r >= (rank_bad ? 0 : nj) && r < ni) rr = fma(bv[r], bv[r], rr);
                }
                rr = wsum(rr) + bo2;
                if (lane == 0) a.colres[j] = sqrt(rr);
            }
            if (lane == 0 && a.steps) a.steps[j] = 0;
        } else {
            // ---------------- MR iteration (Algorithms 2 / 4) ----------------
            const double alpha0 = *a.alpha0;
            if (lane < nj) {
                const int32_t rowc = Jcol[lane];
                const int p = find_row(Irow, ni, rowc);
                Jpos[lane] = p;
                xs[lane] = rowc == j ? alpha0 : 0.0;          // m = alpha0 e_j on the pattern
                double bo = 0.0;                              // b at a row J_c outside I_j
                if (p < 0) {
                    if (a.Aold) {
                        for (int64_t e = a.Acp[j]; e < a.Acp[j + 1]; ++e)
                            if (a.Ari[e] == rowc) bo = a.Aold[a.Atp[e]];
                    } else {
                        bo = rowc == j ? 1.0 : 0.0;
                    }
                }
                bout[lane] = bo;
            }
            __syncwarp();
            // r = b - Ah m on I_j (rows outside keep b)
            double rloc[R], bb = 0.0, rn2 = 0.0;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int r = lane + 32 * q;
                double am = 0.0;
                for (int c = 0; c < nj; ++c) am = fma(Ah[c * kLd + r], xs[c], am);
                const double b = bv[r];
                rloc[q] = r < ni ? b - am : 0.0;
                bb = fma(b, b, bb);
                rn2 = fma(rloc[q], rloc[q], rn2);
            }
            bb = wsum(bb) + bo2;
            rn2 = wsum(rn2) + bo2;
            const double thr2 = a.relative ? (a.tol * a.tol) * bb : a.tol * a.tol;
            int k = 0;
            while (rn2 > thr2 && k < a.kmax) {
                // d = r restricted to the pattern J_j
                for (int c = 0; c < nj; ++c) {
                    const int p = Jpos[c];                    // the same in every lane
                    double d;
                    if (p >= 0) {
                        double src = rloc[0];                 // row p lives in lane p & 31, slot p >> 5
#pragma unroll
                        for (int q = 1; q < R; ++q)
                            if ((p >> 5) == q) src = rloc[q];
                        d = __shfl_sync(0xffffffffu, src, p & 31);
                    } else {
                        d = bout[c];
                    }
                    if (lane == 0) dv[c] = d;
                }
                __syncwarp();
                double w[R], ww = 0.0, rw = 0.0;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int r = lane + 32 * q;
                    double s = 0.0;
                    for (int c = 0; c < nj; ++c) s = fma(Ah[c * kLd + r], dv[c], s);
                    w[q] = s;
                    ww = fma(s, s, ww);
                    rw = fma(rloc[q], s, rw);
                }
                ww = wsum(ww);
                rw = wsum(rw);
                if (ww == 0.0) break;                         // r vanishes on the pattern
                const double al = rw / ww;
                if (lane < nj) xs[lane] = fma(al, dv[lane], xs[lane]);
                rn2 = 0.0;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    rloc[q] = fma(-al, w[q], rloc[q]);
                    rn2 = fma(rloc[q], rloc[q], rn2);
                }
                rn2 = wsum(rn2) + bo2;
                ++k;
                __syncwarp();
            }
            if (lane == 0) {
                if (a.steps) a.steps[j] = k;
                if (a.colres) a.colres[j] = sqrt(rn2);
            }
        }
        __syncwarp();
        if (lane < nj) {
            const int64_t t = a.Stp[sb + lane];
            if (AIRGA_CK(t, 0, a.nnz_s, 407)) a.F[t] = xs[lane];
        }
        __syncwarp();
    }
}

}  // namespace

int csr_spai_rows(const CsrPatPtr &A, const CsrPatPtr &S, cudaStream_t s,
                  const CsrPat::Rows **out) {
    for (auto &r : A->spai_rows) {
        auto sp = r.S.lock();
        if (sp && sp.get() == S.get()) {
            *out = &r;
            return AIRGA_OK;
        }
    }
    const int64_t n = A->n;
    std::shared_ptr<void> cntb;
    int st = make_buf(sizeof(int64_t) * (size_t)(n + 1) + 4 * sizeof(int32_t), s, &cntb);
    if (st) return st;
    int64_t *cnt = (int64_t *)cntb.get();
    int32_t *stats = (int32_t *)(cnt + (n + 1));
    AIRGA_CUDA(cudaMemsetAsync(cntb.get(), 0, sizeof(int64_t) * (size_t)(n + 1) + 4 * sizeof(int32_t), s));
    int dev = 0, sms = 152;
    AIRGA_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + kRowsWarps - 1) / kRowsWarps;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    spai_rows_kernel<false><<<(unsigned)blocks, 32 * kRowsWarps, 0, s>>>(
        n, A->colptr, A->rowidx, S->colptr, S->rowidx, cnt, nullptr, nullptr, stats);
    AIRGA_CUDA(cudaGetLastError());
    scan_kernel<<<1, 1024, 0, s>>>(cnt, n + 1);
    AIRGA_CUDA(cudaGetLastError());
    int32_t hs[4] = {0, 0, 0, 0};
    int64_t total = 0;
    AIRGA_CUDA(cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    AIRGA_CUDA(cudaMemcpyAsync(&total, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AIRGA_CUDA(cudaStreamSynchronize(s));
    if (hs[2] & 1)
        return fail(AIRGA_E_INVALID_ARG, "spai: a pattern column has more than 32 entries");
    if (hs[2] & 6)
        return fail(AIRGA_E_INVALID_ARG,
                    "spai: a column's least-squares block touches more than 64 rows of A");
    std::shared_ptr<void> rows;
    st = make_buf(sizeof(int32_t) * (size_t)(total + 1), s, &rows);
    if (st) return st;
    spai_rows_kernel<true><<<(unsigned)blocks, 32 * kRowsWarps, 0, s>>>(
        n, A->colptr, A->rowidx, S->colptr, S->rowidx, nullptr, cnt, (int32_t *)rows.get(), nullptr);
    AIRGA_CUDA(cudaGetLastError());
    struct Both {
        std::shared_ptr<void> a, b;
    };
    auto both = std::make_shared<Both>(Both{cntb, rows});
    CsrPat::Rows r;
    r.S = S;
    r.buf = std::shared_ptr<void>(both, both.get());
    r.iptr = cnt;
    r.irows = (const int32_t *)rows.get();
    r.max_i = hs[0];
    r.max_j = hs[1];
    A->spai_rows.push_back(r);
    *out = &A->spai_rows.back();
    return AIRGA_OK;
}

cudaError_t launch_spai_csr(const CsrPat &A, const double *Av, const double *Aold,
                            const CsrPat &S, const CsrPat::Rows &rows, int mr,
                            const double *alpha0, double tol, int relative, int kmax, double *F,
                            int32_t *steps, double *colres, int32_t *flag, cudaStream_t s) {
    const cudaError_t fe = injected_launch_error();   // host-side test fault only
    if (fe != cudaSuccess) return fe;
    SpaiCsrArgs a;
    a.n = A.n;
    a.nnz_a = A.nnz;
    a.nnz_s = S.nnz;
    a.Acp = A.colptr;
    a.Ari = A.rowidx;
    a.Atp = A.tperm;
    a.Av = Av;
    a.Aold = Aold;
    a.Scp = S.colptr;
    a.Sri = S.rowidx;
    a.Stp = S.tperm;
    a.iptr = rows.iptr;
    a.irows = rows.irows;
    a.mr = mr;
    a.alpha0 = alpha0;
    a.tol = tol;
    a.relative = relative;
    a.kmax = kmax;
    a.F = F;
    a.steps = steps;
    a.colres = colres;
    a.flag = flag;
    const int max_j = rows.max_j > 0 ? rows.max_j : 1;
    int dev = 0, sms = 152;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (A.n + kNumWarps - 1) / kNumWarps;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    if (rows.max_i <= 32) {
        const size_t smem = kNumWarps * WarpMem<1>::bytes(max_j);
        e = cudaFuncSetAttribute(spai_csr_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        spai_csr_kernel<1><<<(unsigned)blocks, 32 * kNumWarps, smem, s>>>(a, max_j);
    } else {
        const size_t smem = kNumWarps * WarpMem<2>::bytes(max_j);
        e = cudaFuncSetAttribute(spai_csr_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        spai_csr_kernel<2><<<(unsigned)blocks, 32 * kNumWarps, smem, s>>>(a, max_j);
    }
    return cudaGetLastError();
}

}  // namespace airga

AIRGA_CHECK_READER(spai_csr)
