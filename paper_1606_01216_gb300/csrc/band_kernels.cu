// Band-7 kernels: CSR import, shifted assembly, mat-vecs, symmetrisation,
// true residual and the MR initial-scaling reductions.
//
// Storage: band[(d+3)*n + i] = A(i, i+d), d = -3..3 (diagonal-major SoA, so
// consecutive threads = consecutive rows read consecutive addresses of each
// diagonal).  Entries outside the matrix are stored as 0 and never read
// against out-of-range vector entries.
//
// GB300 note: the FP64 pipe issues 2 FMA/clk/SM (about 1.2 TFLOP/s for the
// whole chip) while HBM3e streams about 6.7 TB/s, so even these "streaming"
// kernels sit near the FP64/HBM ridge (~0.18 flop/B).  Every kernel below
// keeps its FP64 operation count at the minimum the formula needs.
#include "airga_internal.cuh"
#include "ieee_conv.cuh"

namespace airga {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int threads = kThreads) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 8;   // 8 resident 256-thread CTAs per SM
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// ---------------------------------------------------------------------------
// CSR -> band-7.  One thread per row: zero the row's 7 slots, then add each
// stored entry to its diagonal (duplicates sum).  flag bit 1: an entry with
// |col - row| > 3; bit 2: a column outside [0, n) or a decreasing rowptr.
// ---------------------------------------------------------------------------
__global__ void csr_to_band_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                   const int32_t *__restrict__ col,
                                   const double *__restrict__ val, double *__restrict__ band,
                                   int32_t *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc[kBand];
#pragma unroll
        for (int d = 0; d < kBand; ++d) acc[d] = 0.0;
        int64_t b = rowptr[i], e = rowptr[i + 1];
        int bad = 0;
        if (e < b) bad |= 2;
        for (int64_t k = b; k < e; ++k) {
            int64_t c = col[k];
            if (c < 0 || c >= n) { bad |= 2; continue; }
            int64_t d = c - i;
            if (d < -kHalf || d > kHalf) { bad |= 1; continue; }
            // unrolled select keeps acc[] in registers
#pragma unroll
            for (int q = 0; q < kBand; ++q)
                if (q == d + kHalf) acc[q] += val[k];
        }
#pragma unroll
        for (int d = 0; d < kBand; ++d) band[d * n + i] = acc[d];
        if (bad) atomicOr(flag, bad);
    }
}

// ---------------------------------------------------------------------------
// A = cm M + ck K, cm = s^2 + alpha s, ck = 1 + beta s: the coefficient
// matrix s^2 M + s (alpha M + beta K) + K with the two scalar weights folded
// on the host, so each stored entry costs one FP64 multiply and one FMA.
// double2 loads/stores over the whole 7n band (7n is even when n is even;
// the odd tail is handled separately).
// ---------------------------------------------------------------------------
__global__ void assemble_kernel(int64_t total, const double *__restrict__ M,
                                const double *__restrict__ K, double cm, double ck,
                                double *__restrict__ A, const int32_t *fm, const int32_t *fk,
                                int32_t *fa) {
    // a zero of both M and K stays an exact zero of A: the structure flag of
    // A is the AND of the two input flags
    if (fa && blockIdx.x == 0 && threadIdx.x == 0) *fa = (fm && fk && *fm && *fk) ? 1 : 0;
    int64_t pairs = total >> 1;
    const double2 *M2 = reinterpret_cast<const double2 *>(M);
    const double2 *K2 = reinterpret_cast<const double2 *>(K);
    double2 *A2 = reinterpret_cast<double2 *>(A);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 m = __ldcs(M2 + i), k = __ldcs(K2 + i);
        double2 a;
        a.x = fma(cm, m.x, ck * k.x);
        a.y = fma(cm, m.y, ck * k.y);
        __stcs(A2 + i, a);
    }
    if ((total & 1) && blockIdx.x == 0 && threadIdx.x == 0)
        A[total - 1] = fma(cm, M[total - 1], ck * K[total - 1]);
}

// The same assembly by row pairs (n even), also writing the packed beam
// nonzeros of A (layout of pack_pairs_kernel) when both inputs carry the beam
// zero-structure flag: the CG kernel's packed stencil then needs no separate
// packing pass over A.  Thread j owns rows (2j, 2j+1): seven double2 loads
// of M and of K, seven double2 stores of A and, for a beam, five double2
// stores of the packed entries (even row offsets -2,-1,0,2,3, odd row
// -3,-2,0,1,2).
__global__ void assemble_pack_kernel(int64_t n, const double *__restrict__ M,
                                     const double *__restrict__ K, double cm, double ck,
                                     double *__restrict__ A, double *__restrict__ packed,
                                     const int32_t *fm, const int32_t *fk, int32_t *fa) {
    const bool beam = fm && fk && *fm && *fk;
    if (fa && blockIdx.x == 0 && threadIdx.x == 0) *fa = beam ? 1 : 0;
    const int64_t pairs = n >> 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < pairs;
         j += (int64_t)gridDim.x * blockDim.x) {
        double2 a[kBand];
#pragma unroll
        for (int d = 0; d < kBand; ++d) {
            const int64_t o = (int64_t)d * (n >> 1) + j;      // double2 index of rows (2j, 2j+1)
            const double2 m = __ldcs(reinterpret_cast<const double2 *>(M) + o);
            const double2 k = __ldcs(reinterpret_cast<const double2 *>(K) + o);
            a[d].x = fma(cm, m.x, ck * k.x);
            a[d].y = fma(cm, m.y, ck * k.y);
            __stcs(reinterpret_cast<double2 *>(A) + o, a[d]);
        }
        if (beam) {
            // band index = offset + 3; even row (x): 1,2,3,5,6; odd row (y): 0,1,3,4,5
            double2 *P2 = reinterpret_cast<double2 *>(packed);
            const int64_t h = n >> 1;
            P2[0 * h + j] = make_double2(a[1].x, a[0].y);
            P2[1 * h + j] = make_double2(a[2].x, a[1].y);
            P2[2 * h + j] = make_double2(a[3].x, a[3].y);
            P2[3 * h + j] = make_double2(a[5].x, a[4].y);
            P2[4 * h + j] = make_double2(a[6].x, a[5].y);
        }
    }
}

// Beam zero structure: every row pair (2k, 2k+1) except the last has exact
// zeros at offsets -3, +1 (even row) and +3, -1 (odd row).  `flag` arrives
// nonzero; any violation clears it (all writers store the same 0).
__global__ void detect_pairz_kernel(int64_t n, const double *__restrict__ band, int32_t *flag) {
    if (n < 2 || (n & 1)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0;
        return;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 2;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool bad = (i & 1) ? (band[6 * n + i] != 0.0 || band[2 * n + i] != 0.0)
                                 : (band[0 * n + i] != 0.0 || band[4 * n + i] != 0.0);
        if (bad) *flag = 0;
    }
}

// Packed nonzeros of the beam row pairs: for pair (i, i+1), slot k holds the
// even row's offset dE[k] and the odd row's offset dO[k].
__global__ void pack_pairs_kernel(int64_t n, const double *__restrict__ band,
                                  double *__restrict__ packed) {
    const int dE[5] = {-2, -1, 0, 2, 3};
    const int dO[5] = {-3, -2, 0, 1, 2};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = 2 * j;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            packed[k * n + i] = band[(dE[k] + kHalf) * n + i];
            packed[k * n + i + 1] = band[(dO[k] + kHalf) * n + i + 1];
        }
    }
}

// one row of y = A x for the band-7 stencil (x read through a bounds check)
__device__ __forceinline__ double band_row(const double *__restrict__ band, int64_t n, int64_t i,
                                           const double *__restrict__ x) {
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < kBand; ++d) {
        int64_t c = i + d - kHalf;
        if (c >= 0 && c < n) acc = fma(band[d * n + i], x[c], acc);
    }
    return acc;
}

// one row of y = A^T x: (A^T x)_i = sum_d A(i+d, i) x_{i+d},
// A(i+d, i) = band[(3-d)*n + i+d]
__device__ __forceinline__ double band_row_t(const double *__restrict__ band, int64_t n,
                                             int64_t i, const double *__restrict__ x) {
    double acc = 0.0;
#pragma unroll
    for (int d = -kHalf; d <= kHalf; ++d) {
        int64_t c = i + d;
        if (c >= 0 && c < n) acc = fma(band[(kHalf - d) * n + c], x[c], acc);
    }
    return acc;
}

__global__ void spmv_kernel(int64_t n, const double *__restrict__ band,
                            const double *__restrict__ X, double *__restrict__ Y, int32_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int32_t c = 0; c < m; ++c) Y[c * n + i] = band_row(band, n, i, X + c * n);
}

__global__ void band_apply_kernel(int64_t n, const double *__restrict__ band,
                                  const double *__restrict__ x, double *__restrict__ y,
                                  int transpose) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = transpose ? band_row_t(band, n, i, x) : band_row(band, n, i, x);
}

// Psym(i, i+d) = 1/2 (P(i, i+d) + P(i+d, i)); P(i+d, i) = band[(3-d)*n + i+d].
// Thread i forms each of its pairs d = 1..3 once and writes both mirrored
// entries (i, i+d) and (i+d, i); the diagonal is copied.  One FP64 add per
// pair and an exact integer halving (ieee::half_of, = x / 2 bit for bit) —
// on GB300 the FP64 pipe, not HBM, bound the one-entry-per-thread form.
__global__ void symmetrize_kernel(int64_t n, const double *__restrict__ P,
                                  double *__restrict__ S) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        S[kHalf * n + i] = P[kHalf * n + i];
#pragma unroll
        for (int d = 1; d <= kHalf; ++d) {
            if (i + d < n) {
                const double v = ieee::half_of(P[(kHalf + d) * n + i] + P[(kHalf - d) * n + i + d]);
                S[(kHalf + d) * n + i] = v;             // (i, i+d)
                S[(kHalf - d) * n + i + d] = v;         // (i+d, i)
            } else {
                S[(kHalf + d) * n + i] = 0.0;           // column outside the matrix
            }
            if (i < d) S[(kHalf - d) * n + i] = 0.0;    // column i-d outside the matrix
        }
    }
}

__global__ void axpby_kernel(int64_t n, double a, const double *__restrict__ x, double b,
                             double *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], b * y[i]);
}

// ---------------------------------------------------------------------------
// deterministic block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of v over the block, valid in thread 0
__device__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
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

// per-block partial ||F_c - A X_c||^2 and ||F_c||^2 (fixed block partition)
__global__ void resid_partial_kernel(int64_t n, const double *__restrict__ band,
                                     const double *__restrict__ X,
                                     const double *__restrict__ F, int32_t m,
                                     double *__restrict__ partial) {
    __shared__ double sh[32];
    int64_t per = (n + gridDim.x - 1) / gridDim.x;
    int64_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
    for (int32_t c = 0; c < m; ++c) {
        double rr = 0.0, ff = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            double f = F[c * n + i];
            double r = f - band_row(band, n, i, X + c * n);
            rr = fma(r, r, rr);
            ff = fma(f, f, ff);
        }
        double srr = block_sum(rr, sh);
        double sff = block_sum(ff, sh);
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
        double srr = block_sum(rr, sh);
        double sff = block_sum(ff, sh);
        if (threadIdx.x == 0) relres[c] = sff > 0.0 ? sqrt(srr) / sqrt(sff) : 0.0;
    }
}

// MR initial scalings (Algorithm 2 line 2; Sec. 3.2):
//   build : t0 = trace(A),           t1 = trace(A A^T) = sum of squares
//   update: t0 = <A_old, A_new>_F  (= 1/2 trace(A_old^T A_new + A_new^T A_old)),
//           t1 = trace(A_new^T A_new)
__global__ void mr_alpha_partial_kernel(int64_t n, const double *__restrict__ A,
                                        const double *__restrict__ Aold,
                                        double *__restrict__ partial) {
    __shared__ double sh[32];
    int64_t total = (int64_t)kBand * n;
    int64_t per = (total + gridDim.x - 1) / gridDim.x;
    int64_t lo = blockIdx.x * per, hi = lo + per < total ? lo + per : total;
    double t0 = 0.0, t1 = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        double a = A[e];
        t1 = fma(a, a, t1);
        if (Aold) t0 = fma(Aold[e], a, t0);
        else if (e >= kHalf * n && e < (kHalf + 1) * n) t0 += a;   // main diagonal
    }
    double s0 = block_sum(t0, sh);
    double s1 = block_sum(t1, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s0;
        partial[gridDim.x + blockIdx.x] = s1;
    }
}

__global__ void mr_alpha_final_kernel(int nblk, const double *__restrict__ partial,
                                      double *__restrict__ out) {
    __shared__ double sh[32];
    double t0 = 0.0, t1 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        t0 += partial[b];
        t1 += partial[nblk + b];
    }
    double s0 = block_sum(t0, sh);
    double s1 = block_sum(t1, sh);
    if (threadIdx.x == 0) {
        out[0] = s0;
        out[1] = s1;
        out[2] = s0 / s1;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_csr_to_band(int64_t n, const int64_t *rowptr, const int32_t *col,
                               const double *val, double *band, int32_t *flag, cudaStream_t s) {
    csr_to_band_kernel<<<grid_for(n), kThreads, 0, s>>>(n, rowptr, col, val, band, flag);
    return cudaGetLastError();
}

cudaError_t launch_assemble_pack(int64_t n, const double *M, const double *K, double alpha,
                                 double beta, double sh, double *A, double *packed, cudaStream_t s,
                                 const int32_t *fm, const int32_t *fk, int32_t *fa) {
    const double cm = sh * sh + alpha * sh;
    const double ck = 1.0 + beta * sh;
    assemble_pack_kernel<<<grid_for(n / 2 + 1), kThreads, 0, s>>>(n, M, K, cm, ck, A, packed, fm,
                                                                   fk, fa);
    return cudaGetLastError();
}

cudaError_t launch_assemble(int64_t n, const double *M, const double *K, double alpha,
                            double beta, double sh, double *A, cudaStream_t s,
                            const int32_t *fm, const int32_t *fk, int32_t *fa) {
    double cm = sh * sh + alpha * sh;
    double ck = 1.0 + beta * sh;
    int64_t total = (int64_t)kBand * n;
    assemble_kernel<<<grid_for(total / 2 + 1), kThreads, 0, s>>>(total, M, K, cm, ck, A, fm, fk,
                                                                   fa);
    return cudaGetLastError();
}

cudaError_t launch_pack_pairs(int64_t n, const double *band, double *packed, cudaStream_t s) {
    pack_pairs_kernel<<<grid_for(n / 2 + 1), kThreads, 0, s>>>(n, band, packed);
    return cudaGetLastError();
}

cudaError_t launch_detect_pairz(int64_t n, const double *band, int32_t *flag, cudaStream_t s) {
    detect_pairz_kernel<<<grid_for(n), kThreads, 0, s>>>(n, band, flag);
    return cudaGetLastError();
}

cudaError_t launch_spmv(int64_t n, const double *band, const double *X, double *Y, int32_t m,
                        cudaStream_t s) {
    spmv_kernel<<<grid_for(n), kThreads, 0, s>>>(n, band, X, Y, m);
    return cudaGetLastError();
}

cudaError_t launch_band_apply(int64_t n, const double *band, const double *x, double *y,
                              bool transpose, cudaStream_t s) {
    band_apply_kernel<<<grid_for(n), kThreads, 0, s>>>(n, band, x, y, transpose ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(int64_t n, const double *P, double *Psym, cudaStream_t s) {
    symmetrize_kernel<<<grid_for(n), kThreads, 0, s>>>(n, P, Psym);
    return cudaGetLastError();
}

cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y,
                         cudaStream_t s) {
    axpby_kernel<<<grid_for(n), kThreads, 0, s>>>(n, a, x, b, y);
    return cudaGetLastError();
}

int true_residual_blocks(int64_t n) {
    int64_t b = (n + 4095) / 4096;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

cudaError_t launch_true_residual(int64_t n, const double *band, const double *X,
                                 const double *F, int32_t m, double *relres, double *partial,
                                 int nblk, cudaStream_t s) {
    resid_partial_kernel<<<nblk, kThreads, 0, s>>>(n, band, X, F, m, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resid_final_kernel<<<1, kThreads, 0, s>>>(nblk, m, partial, relres);
    return cudaGetLastError();
}

int mr_alpha_blocks(int64_t n) {
    int64_t b = ((int64_t)kBand * n + 8191) / 8192;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

cudaError_t launch_mr_alpha(int64_t n, const double *A, const double *A_old, double *partial,
                            int nblk, double *out, cudaStream_t s) {
    mr_alpha_partial_kernel<<<nblk, kThreads, 0, s>>>(n, A, A_old, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mr_alpha_final_kernel<<<1, kThreads, 0, s>>>(nblk, partial, out);
    return cudaGetLastError();
}

}  // namespace airga
