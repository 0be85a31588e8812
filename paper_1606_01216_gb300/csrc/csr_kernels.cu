// General sparse (CSR) storage: import and canonicalisation, the transposed
// structure, sparse sums, mat-vecs, the true residual and the MR initial
// scalings, for matrices whose entries leave the band |i - j| <= 3 (the
// paper's M, D and K are general sparse matrices, Eq. 1.1; the SPAI pattern
// S of Eq. 3.1 is an input).
//
// Every structural step runs on the device: per-row insertion sort (rows of
// finite-element matrices are short), duplicate summation in input order, a
// single-CTA tiled prefix sum, an atomic scatter into the transposed
// structure followed by a per-column sort (so the result does not depend on
// the order of the atomics).  The host reads back only sizes and the
// longest row / column, at pattern creation.
#include "csr_common.cuh"

namespace airga {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int threads = kThreads) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 8;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

#define GRID_STRIDE(i, count)                                                          \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (count); \
         i += (int64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// prefix sums
// ---------------------------------------------------------------------------

// In-place inclusive scan of a[0..len) by one CTA of 1024 threads, tile by
// tile (8 values per thread), carrying the running total between tiles.
__global__ void __launch_bounds__(1024) scan_inclusive_kernel(int64_t *a, int64_t len) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    constexpr int kPer = 8;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 1024 * kPer) {
        int64_t v[kPer];
        int64_t t = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t idx = base + (int64_t)tid * kPer + k;
            v[k] = idx < len ? a[idx] : 0;
            t += v[k];
            v[k] = t;                                   // inclusive within the thread
        }
        // inclusive scan of the thread totals within the warp
        int64_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;                             // inclusive warp prefix
        }
        __syncthreads();
        const int64_t before = carry + (w > 0 ? wsum[w - 1] : 0) + (x - t);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t idx = base + (int64_t)tid * kPer + k;
            if (idx < len) a[idx] = before + v[k];
        }
        __syncthreads();
        if (tid == 0) carry += wsum[31];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// canonical CSR from the caller's arrays
// ---------------------------------------------------------------------------

// Copy row i's entries (input base rowptr[0]) to position rowptr[i] - rowptr[0]
// of the work arrays and sort them by column (insertion sort, stable, so
// duplicates keep their input order); cnt[i + 1] = number of distinct columns.
__global__ void csr_sort_rows_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                     const int32_t *__restrict__ col,
                                     const double *__restrict__ val, int32_t *__restrict__ wcol,
                                     double *__restrict__ wval, int64_t *__restrict__ cnt) {
    const int64_t base = rowptr[0];
    GRID_STRIDE(i, n) {
        const int64_t b = rowptr[i] - base, e = rowptr[i + 1] - base;
        for (int64_t k = b; k < e; ++k) {
            const int32_t c = col[k + base];
            const double v = val[k + base];
            int64_t q = k;
            while (q > b && wcol[q - 1] > c) {
                wcol[q] = wcol[q - 1];
                wval[q] = wval[q - 1];
                --q;
            }
            wcol[q] = c;
            wval[q] = v;
        }
        int64_t u = 0;
        for (int64_t k = b; k < e; ++k) u += (k == b || wcol[k] != wcol[k - 1]) ? 1 : 0;
        cnt[i + 1] = u;
    }
}

// Distinct columns of each sorted row, duplicates summed in input order.
__global__ void csr_compact_kernel(int64_t n, const int64_t *__restrict__ rowptr_in,
                                   const int32_t *__restrict__ wcol,
                                   const double *__restrict__ wval,
                                   const int64_t *__restrict__ rowptr, int32_t *__restrict__ col,
                                   double *__restrict__ val) {
    const int64_t base = rowptr_in[0];
    GRID_STRIDE(i, n) {
        const int64_t b = rowptr_in[i] - base, e = rowptr_in[i + 1] - base;
        int64_t o = rowptr[i] - 1;
        for (int64_t k = b; k < e; ++k) {
            if (k == b || wcol[k] != wcol[k - 1]) {
                ++o;
                col[o] = wcol[k];
                val[o] = wval[k];
            } else {
                val[o] += wval[k];
            }
        }
    }
}

// flag bit 1: an entry with |col - row| > 3; bit 2: malformed (rowptr[0] != 0,
// rowptr[n] != nnz, a decreasing rowptr, a column outside [0, n)).  Reads stay
// inside [0, nnz) of col whatever rowptr holds.
__global__ void csr_validate_kernel(int64_t n, int64_t nnz, const int64_t *__restrict__ rowptr,
                                    const int32_t *__restrict__ col, int32_t *flag) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || rowptr[n] != nnz))
        atomicOr(flag, 2);
    GRID_STRIDE(i, n) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        int bad = 0;
        if (b < 0 || e > nnz || e < b) {
            bad = 2;
        } else {
            for (int64_t k = b; k < e; ++k) {
                const int64_t c = col[k];
                if (c < 0 || c >= n) bad |= 2;
                else if (c - i < -kHalf || c - i > kHalf) bad |= 1;
            }
        }
        if (bad) atomicOr(flag, bad);
    }
}

// ---------------------------------------------------------------------------
// transposed structure
// ---------------------------------------------------------------------------

__global__ void count_cols_kernel(int64_t nnz, const int32_t *__restrict__ col,
                                  unsigned long long *__restrict__ colcnt) {
    GRID_STRIDE(e, nnz) atomicAdd(colcnt + col[e] + 1, 1ull);
}

__global__ void scatter_cols_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                    const int32_t *__restrict__ col,
                                    unsigned long long *__restrict__ cursor,
                                    int32_t *__restrict__ rowidx, int64_t *__restrict__ tperm) {
    GRID_STRIDE(i, n) {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int64_t f = (int64_t)atomicAdd(cursor + col[e], 1ull);
            rowidx[f] = (int32_t)i;
            tperm[f] = e;
        }
    }
}

// Sort each column's entries by row (rows are distinct within a column).
__global__ void sort_cols_kernel(int64_t n, const int64_t *__restrict__ colptr,
                                 int32_t *__restrict__ rowidx, int64_t *__restrict__ tperm) {
    GRID_STRIDE(j, n) {
        const int64_t b = colptr[j], e = colptr[j + 1];
        for (int64_t k = b + 1; k < e; ++k) {
            const int32_t r = rowidx[k];
            const int64_t t = tperm[k];
            int64_t q = k;
            while (q > b && rowidx[q - 1] > r) {
                rowidx[q] = rowidx[q - 1];
                tperm[q] = tperm[q - 1];
                --q;
            }
            rowidx[q] = r;
            tperm[q] = t;
        }
    }
}

// stats[0] = longest row, stats[1] = longest column, stats[2] = 1 while the
// CSC arrays equal the CSR arrays (structural symmetry), preset to 1.
__global__ void pattern_stats_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                     const int32_t *__restrict__ col,
                                     const int64_t *__restrict__ colptr,
                                     const int32_t *__restrict__ rowidx, int32_t *stats) {
    int32_t mr = 0, mc = 0;
    bool sym = true;
    GRID_STRIDE(i, n) {
        const int64_t b = rowptr[i], e = rowptr[i + 1];
        mr = max(mr, (int32_t)(e - b));
        mc = max(mc, (int32_t)(colptr[i + 1] - colptr[i]));
        if (colptr[i + 1] != e) {
            sym = false;
        } else {
            for (int64_t k = b; k < e; ++k)
                if (rowidx[k] != col[k]) { sym = false; break; }
        }
    }
    atomicMax(stats, mr);
    atomicMax(stats + 1, mc);
    if (!sym) atomicExch(stats + 2, 0);
}

// ---------------------------------------------------------------------------
// band <-> CSR
// ---------------------------------------------------------------------------

// Entries of the full band |i - j| <= 3 in rows 0..i-1 of an n x n matrix:
// row k holds 7 - max(0, 3 - k) - max(0, k + 3 - (n - 1)) of them.
__device__ __forceinline__ int64_t band_entries_before(int64_t n, int64_t i) {
    int64_t cut = 0;
    for (int64_t k = 0; k < 3 && k < i; ++k) cut += 3 - k;                      // left edge
    for (int64_t k = n - 3 > 0 ? n - 3 : 0; k < i; ++k) cut += k + 3 - (n - 1);  // right edge
    return 7 * i - cut;
}

// CSR pattern of the full band |i - j| <= 3 inside the matrix
__global__ void band_pattern_kernel(int64_t n, int64_t *__restrict__ rowptr,
                                    int32_t *__restrict__ col) {
    GRID_STRIDE(i, n + 1) {
        const int64_t before = band_entries_before(n, i);
        rowptr[i] = before;
        if (i < n) {
            int64_t o = before;
            for (int d = -kHalf; d <= kHalf; ++d) {
                const int64_t c = i + d;
                if (c >= 0 && c < n) col[o++] = (int32_t)c;
            }
        }
    }
}

// nonzero entries of a band-7 array: cnt[i + 1] = count of row i, then the
// sorted columns and values
__global__ void band_nz_count_kernel(int64_t n, const double *__restrict__ band,
                                     int64_t *__restrict__ cnt) {
    GRID_STRIDE(i, n) {
        int64_t c = 0;
        for (int d = -kHalf; d <= kHalf; ++d) {
            const int64_t j = i + d;
            if (j >= 0 && j < n && band[(int64_t)(d + kHalf) * n + i] != 0.0) ++c;
        }
        cnt[i + 1] = c;
    }
}

__global__ void band_nz_fill_kernel(int64_t n, const double *__restrict__ band,
                                    const int64_t *__restrict__ rowptr, int32_t *__restrict__ col,
                                    double *__restrict__ val) {
    GRID_STRIDE(i, n) {
        int64_t o = rowptr[i];
        for (int d = -kHalf; d <= kHalf; ++d) {
            const int64_t j = i + d;
            const double v = (j >= 0 && j < n) ? band[(int64_t)(d + kHalf) * n + i] : 0.0;
            if (v != 0.0) {
                col[o] = (int32_t)j;
                val[o] = v;
                ++o;
            }
        }
    }
}

// flag = 1 where two patterns of equal n and nnz differ
__global__ void same_structure_kernel(int64_t n, int64_t nnz, const int64_t *__restrict__ ra,
                                      const int32_t *__restrict__ ca, const int64_t *__restrict__ rb,
                                      const int32_t *__restrict__ cb, int32_t *flag) {
    GRID_STRIDE(i, n + 1) if (ra[i] != rb[i]) atomicExch(flag, 1);
    GRID_STRIDE(e, nnz) if (ca[e] != cb[e]) atomicExch(flag, 1);
}

__global__ void band_values_kernel(int64_t n, const double *__restrict__ band,
                                   const int64_t *__restrict__ rowptr, double *__restrict__ val) {
    GRID_STRIDE(i, n) {
        int64_t o = rowptr[i];
        for (int d = -kHalf; d <= kHalf; ++d) {
            const int64_t c = i + d;
            if (c >= 0 && c < n) val[o++] = band[(int64_t)(d + kHalf) * n + i];
        }
    }
}

// ---------------------------------------------------------------------------
// sparse sums Z = a X + b Y on the union pattern (rows merged by column)
// ---------------------------------------------------------------------------

__global__ void union_count_kernel(int64_t n, RowView X, RowView Y, int64_t *__restrict__ cnt) {
    GRID_STRIDE(i, n) {
        int64_t p = X.ptr[i], pe = X.ptr[i + 1], q = Y.ptr[i], qe = Y.ptr[i + 1], u = 0;
        while (p < pe || q < qe) {
            const int32_t cx = p < pe ? X.idx[p] : INT32_MAX, cy = q < qe ? Y.idx[q] : INT32_MAX;
            if (cx <= cy) ++p;
            if (cy <= cx) ++q;
            ++u;
        }
        cnt[i + 1] = u;
    }
}

__global__ void union_cols_kernel(int64_t n, RowView X, RowView Y, const int64_t *__restrict__ rowptr,
                                  int32_t *__restrict__ col) {
    GRID_STRIDE(i, n) {
        int64_t p = X.ptr[i], pe = X.ptr[i + 1], q = Y.ptr[i], qe = Y.ptr[i + 1], o = rowptr[i];
        while (p < pe || q < qe) {
            const int32_t cx = p < pe ? X.idx[p] : INT32_MAX, cy = q < qe ? Y.idx[q] : INT32_MAX;
            col[o++] = cx <= cy ? cx : cy;
            if (cx <= cy) ++p;
            if (cy <= cx) ++q;
        }
    }
}

// Z(i, c) = fma(a, X(i, c), b Y(i, c)), missing entries 0, on Z's pattern.
__global__ void add_values_kernel(int64_t n, double a, RowView X, double b, RowView Y,
                                  const int64_t *__restrict__ rowptr,
                                  const int32_t *__restrict__ col, double *__restrict__ val) {
    GRID_STRIDE(i, n) {
        int64_t p = X.ptr[i], pe = X.ptr[i + 1], q = Y.ptr[i], qe = Y.ptr[i + 1];
        for (int64_t o = rowptr[i]; o < rowptr[i + 1]; ++o) {
            const int32_t c = col[o];
            double x = 0.0, y = 0.0;
            while (p < pe && X.idx[p] < c) ++p;
            while (q < qe && Y.idx[q] < c) ++q;
            if (p < pe && X.idx[p] == c) x = rv_val(X, p);
            if (q < qe && Y.idx[q] == c) y = rv_val(Y, q);
            val[o] = fma(a, x, b * y);
        }
    }
}

// ---------------------------------------------------------------------------
// mat-vecs, true residual, MR scalings
// ---------------------------------------------------------------------------

__global__ void csr_spmv_kernel(int64_t n, RowView A, const double *__restrict__ X,
                                double *__restrict__ Y, int32_t m) {
    GRID_STRIDE(i, n) {
        for (int32_t c = 0; c < m; ++c) Y[(int64_t)c * n + i] = rv_dot(A, i, X + (int64_t)c * n);
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// fixed row partition per block: partial ||F_c - A X_c||^2, ||F_c||^2
__global__ void csr_resid_partial_kernel(int64_t n, RowView A, const double *__restrict__ X,
                                         const double *__restrict__ F, int32_t m,
                                         double *__restrict__ partial) {
    __shared__ double sh[32];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
    for (int32_t c = 0; c < m; ++c) {
        double rr = 0.0, ff = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double f = F[(int64_t)c * n + i];
            const double r = f - rv_dot(A, i, X + (int64_t)c * n);
            rr = fma(r, r, rr);
            ff = fma(f, f, ff);
        }
        const double srr = block_sum(rr, sh);
        const double sff = block_sum(ff, sh);
        if (threadIdx.x == 0) {
            partial[(2 * c) * gridDim.x + blockIdx.x] = srr;
            partial[(2 * c + 1) * gridDim.x + blockIdx.x] = sff;
        }
    }
}

__global__ void resid_final_kernel(int nblk, int32_t m, const double *__restrict__ partial,
                                   double *__restrict__ relres) {
    __shared__ double sh[32];
    for (int32_t c = 0; c < m; ++c) {
        double rr = 0.0, ff = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            rr += partial[(2 * c) * nblk + b];
            ff += partial[(2 * c + 1) * nblk + b];
        }
        const double srr = block_sum(rr, sh);
        const double sff = block_sum(ff, sh);
        if (threadIdx.x == 0) relres[c] = sff > 0.0 ? sqrt(srr) / sqrt(sff) : 0.0;
    }
}

// MR initial scalings over the stored entries (Algorithm 2; Sec. 3.2):
//   build : t0 = trace(A), t1 = trace(A A^T) = sum of squares
//   update: t0 = <A_old, A_new>_F, t1 = ||A_new||_F^2  (A_old on A's pattern)
__global__ void csr_alpha_partial_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                         const int32_t *__restrict__ col,
                                         const double *__restrict__ A,
                                         const double *__restrict__ Aold,
                                         double *__restrict__ partial) {
    __shared__ double sh[32];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
    double t0 = 0.0, t1 = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const double a = A[e];
            t1 = fma(a, a, t1);
            if (Aold) t0 = fma(Aold[e], a, t0);
            else if (col[e] == i) t0 += a;
        }
    }
    const double s0 = block_sum(t0, sh);
    const double s1 = block_sum(t1, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s0;
        partial[gridDim.x + blockIdx.x] = s1;
    }
}

__global__ void alpha_final_kernel(int nblk, const double *__restrict__ partial,
                                   double *__restrict__ out) {
    __shared__ double sh[32];
    double t0 = 0.0, t1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        t0 += partial[b];
        t1 += partial[nblk + b];
    }
    const double s0 = block_sum(t0, sh);
    const double s1 = block_sum(t1, sh);
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s0 / s1;
    }
}

cudaError_t scan_inclusive(int64_t *a, int64_t len, cudaStream_t s) {
    scan_inclusive_kernel<<<1, 1024, 0, s>>>(a, len);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

RowView rows_of(const CsrPat &p, const double *val) {
    return RowView{p.rowptr, p.col, val, nullptr, p.n, p.nnz};
}

RowView cols_of(const CsrPat &p, const double *val) {
    return RowView{p.colptr, p.rowidx, val, p.tperm, p.n, p.nnz};
}

// Pattern from canonical CSR arrays already on the device (rowptr[n+1] with
// rowptr[0] = 0, col[nnz]); `rc` owns them.  Builds the transposed structure
// and reads back the statistics (SYNCHRONISES s).
static int finish_pattern(int64_t n, int64_t nnz, std::shared_ptr<void> rc, int64_t *rowptr,
                          int32_t *col, cudaStream_t s, CsrPatPtr *out) {
    auto p = std::make_shared<CsrPat>();
    p->n = n;
    p->nnz = nnz;
    p->rowptr = rowptr;
    p->col = col;
    std::shared_ptr<void> tm;
    const size_t bytes = sizeof(int64_t) * (size_t)(n + 1) * 2 + sizeof(int32_t) * (size_t)(nnz + 1) +
                         sizeof(int64_t) * (size_t)(nnz + 1) + 64;
    int st = make_buf(bytes, s, &tm);
    if (st) return st;
    char *base = (char *)tm.get();
    p->colptr = (int64_t *)base;
    int64_t *cursor = p->colptr + (n + 1);
    p->tperm = cursor + (n + 1);
    p->rowidx = (int32_t *)(p->tperm + (nnz + 1));
    void *stats_dev = nullptr;
    st = dev_alloc(&stats_dev, 4 * sizeof(int32_t), s);
    if (st) return st;
    int32_t stats[4] = {0, 0, 1, 0};
    cudaError_t e = cudaMemsetAsync(p->colptr, 0, sizeof(int64_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess && nnz > 0) {
        count_cols_kernel<<<grid_for(nnz), kThreads, 0, s>>>(nnz, col, (unsigned long long *)p->colptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_inclusive(p->colptr, n + 1, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cursor, p->colptr, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && nnz > 0) {
        scatter_cols_kernel<<<grid_for(n), kThreads, 0, s>>>(n, rowptr, col,
                                                             (unsigned long long *)cursor, p->rowidx,
                                                             p->tperm);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            sort_cols_kernel<<<grid_for(n), kThreads, 0, s>>>(n, p->colptr, p->rowidx, p->tperm);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(stats_dev, stats, sizeof(stats), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        pattern_stats_kernel<<<grid_for(n), kThreads, 0, s>>>(n, rowptr, col, p->colptr, p->rowidx,
                                                             (int32_t *)stats_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(stats, stats_dev, sizeof(stats), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(stats_dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "csr pattern");
    p->max_row = stats[0];
    p->max_col = stats[1];
    p->symmetric = stats[2] != 0;
    struct Both {
        std::shared_ptr<void> a, b;
    };
    auto both = std::make_shared<Both>(Both{rc, tm});
    p->mem = std::shared_ptr<void>(both, both.get());
    *out = p;
    return AIRGA_OK;
}

int csr_import(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
               const double *val, cudaStream_t s, CsrPatPtr *pat, std::shared_ptr<void> *vals) {
    // work arrays: sorted copy (col, val) and distinct counts
    void *work = nullptr;
    const size_t wbytes = sizeof(int32_t) * (size_t)(nnz + 1) + sizeof(double) * (size_t)(nnz + 1) +
                          sizeof(int64_t) * (size_t)(n + 1) + 64;
    int st = dev_alloc(&work, wbytes, s);
    if (st) return st;
    double *wval = (double *)work;
    int64_t *cnt = (int64_t *)(wval + (nnz + 1));
    int32_t *wcol = (int32_t *)(cnt + (n + 1));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess) {
        csr_sort_rows_kernel<<<grid_for(n), kThreads, 0, s>>>(n, rowptr, col, val, wcol, wval, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_inclusive(cnt, n + 1, s);
    int64_t nnz_u = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz_u, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(work, s);
        return cuda_fail(e, "csr import");
    }
    std::shared_ptr<void> rc, vb;
    st = make_buf(sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz_u + 1) + 16, s, &rc);
    if (!st) st = make_buf(sizeof(double) * (size_t)(nnz_u + 1), s, &vb);
    if (st) {
        dev_free(work, s);
        return st;
    }
    int64_t *rp = (int64_t *)rc.get();
    int32_t *ci = (int32_t *)(rp + (n + 1));
    e = cudaMemcpyAsync(rp, cnt, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        csr_compact_kernel<<<grid_for(n), kThreads, 0, s>>>(n, rowptr, wcol, wval, rp, ci,
                                                            (double *)vb.get());
        e = cudaGetLastError();
    }
    dev_free(work, s);
    if (e != cudaSuccess) return cuda_fail(e, "csr import");
    st = finish_pattern(n, nnz_u, rc, rp, ci, s, pat);
    if (st) return st;
    *vals = vb;
    return AIRGA_OK;
}

cudaError_t launch_csr_validate(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                                int32_t *flag, cudaStream_t s) {
    csr_validate_kernel<<<grid_for(n), kThreads, 0, s>>>(n, nnz, rowptr, col, flag);
    return cudaGetLastError();
}

int band_pattern(int64_t n, cudaStream_t s, CsrPatPtr *out) {
    int64_t nnz = 0;
    for (int64_t d = -kHalf; d <= kHalf; ++d) {
        const int64_t len = n - (d < 0 ? -d : d);
        if (len > 0) nnz += len;
    }
    std::shared_ptr<void> rc;
    int st = make_buf(sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz + 1) + 16, s, &rc);
    if (st) return st;
    int64_t *rp = (int64_t *)rc.get();
    int32_t *ci = (int32_t *)(rp + (n + 1));
    band_pattern_kernel<<<grid_for(n + 1), kThreads, 0, s>>>(n, rp, ci);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "band pattern");
    return finish_pattern(n, nnz, rc, rp, ci, s, out);
}

int band_nonzero_csr(int64_t n, const double *band, cudaStream_t s, CsrPatPtr *pat,
                     std::shared_ptr<void> *vals) {
    void *cnt_v = nullptr;
    int st = dev_alloc(&cnt_v, sizeof(int64_t) * (size_t)(n + 1), s);
    if (st) return st;
    int64_t *cnt = (int64_t *)cnt_v;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess) {
        band_nz_count_kernel<<<grid_for(n), kThreads, 0, s>>>(n, band, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_inclusive(cnt, n + 1, s);
    int64_t nnz = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(cnt_v, s);
        return cuda_fail(e, "band nonzeros");
    }
    std::shared_ptr<void> rc, vb;
    st = make_buf(sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz + 1) + 16, s, &rc);
    if (!st) st = make_buf(sizeof(double) * (size_t)(nnz + 1), s, &vb);
    if (st) {
        dev_free(cnt_v, s);
        return st;
    }
    int64_t *rp = (int64_t *)rc.get();
    int32_t *ci = (int32_t *)(rp + (n + 1));
    e = cudaMemcpyAsync(rp, cnt, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        band_nz_fill_kernel<<<grid_for(n), kThreads, 0, s>>>(n, band, rp, ci, (double *)vb.get());
        e = cudaGetLastError();
    }
    dev_free(cnt_v, s);
    if (e != cudaSuccess) return cuda_fail(e, "band nonzeros");
    st = finish_pattern(n, nnz, rc, rp, ci, s, pat);
    if (st) return st;
    *vals = vb;
    return AIRGA_OK;
}

int csr_same_structure(const CsrPat &a, const CsrPat &b, cudaStream_t s, bool *same) {
    *same = false;
    if (a.n != b.n || a.nnz != b.nnz) return AIRGA_OK;
    void *flag = nullptr;
    int st = dev_alloc(&flag, sizeof(int32_t), s);
    if (st) return st;
    int32_t h = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        same_structure_kernel<<<grid_for(a.nnz > a.n ? a.nnz : a.n + 1), kThreads, 0, s>>>(
            a.n, a.nnz, a.rowptr, a.col, b.rowptr, b.col, (int32_t *)flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(flag, s);
    if (e != cudaSuccess) return cuda_fail(e, "pattern compare");
    *same = h == 0;
    return AIRGA_OK;
}

cudaError_t launch_band_values(const CsrPat &p, const double *band, double *val, cudaStream_t s) {
    band_values_kernel<<<grid_for(p.n), kThreads, 0, s>>>(p.n, band, p.rowptr, val);
    return cudaGetLastError();
}

int csr_union(int64_t n, const RowView &X, const RowView &Y, cudaStream_t s, CsrPatPtr *out) {
    void *cnt_v = nullptr;
    int st = dev_alloc(&cnt_v, sizeof(int64_t) * (size_t)(n + 1), s);
    if (st) return st;
    int64_t *cnt = (int64_t *)cnt_v;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (size_t)(n + 1), s);
    if (e == cudaSuccess) {
        union_count_kernel<<<grid_for(n), kThreads, 0, s>>>(n, X, Y, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_inclusive(cnt, n + 1, s);
    int64_t nnz = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(cnt_v, s);
        return cuda_fail(e, "csr union");
    }
    std::shared_ptr<void> rc;
    st = make_buf(sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz + 1) + 16, s, &rc);
    if (st) {
        dev_free(cnt_v, s);
        return st;
    }
    int64_t *rp = (int64_t *)rc.get();
    int32_t *ci = (int32_t *)(rp + (n + 1));
    e = cudaMemcpyAsync(rp, cnt, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        union_cols_kernel<<<grid_for(n), kThreads, 0, s>>>(n, X, Y, rp, ci);
        e = cudaGetLastError();
    }
    dev_free(cnt_v, s);
    if (e != cudaSuccess) return cuda_fail(e, "csr union");
    return finish_pattern(n, nnz, rc, rp, ci, s, out);
}

cudaError_t launch_csr_add(const CsrPat &Z, double a, const RowView &X, double b,
                           const RowView &Y, double *val, cudaStream_t s) {
    add_values_kernel<<<grid_for(Z.n), kThreads, 0, s>>>(Z.n, a, X, b, Y, Z.rowptr, Z.col, val);
    return cudaGetLastError();
}

cudaError_t launch_csr_spmv(int64_t n, const RowView &A, const double *X, double *Y, int32_t m,
                            cudaStream_t s) {
    csr_spmv_kernel<<<grid_for(n), kThreads, 0, s>>>(n, A, X, Y, m);
    return cudaGetLastError();
}

int csr_blocks(int64_t n) {
    const int64_t b = (n + 2047) / 2048;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

cudaError_t launch_csr_true_residual(int64_t n, const RowView &A, const double *X,
                                     const double *F, int32_t m, double *relres,
                                     double *partial, int nblk, cudaStream_t s) {
    csr_resid_partial_kernel<<<nblk, kThreads, 0, s>>>(n, A, X, F, m, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resid_final_kernel<<<1, kThreads, 0, s>>>(nblk, m, partial, relres);
    return cudaGetLastError();
}

cudaError_t launch_csr_mr_alpha(const CsrPat &p, const double *A, const double *A_old,
                                double *partial, int nblk, double *out, cudaStream_t s) {
    csr_alpha_partial_kernel<<<nblk, kThreads, 0, s>>>(p.n, p.rowptr, p.col, A, A_old, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    alpha_final_kernel<<<1, kThreads, 0, s>>>(nblk, partial, out);
    return cudaGetLastError();
}

}  // namespace airga

AIRGA_CHECK_READER(csr_kernels)
