// Row access to general sparse matrices for the CSR kernels.
//
// A RowView reads row i of a matrix as the entries e in [ptr[i], ptr[i+1])
// with column idx[e] and value val[perm ? perm[e] : e].  The CSR arrays of a
// pattern give the matrix itself; its CSC arrays with the transposition map
// give the transpose (row i of A^T = column i of A) over the same value
// array, so A^T r needs no second copy of the values.
#pragma once

#include "airga_internal.cuh"
#include "check.cuh"

namespace airga {

struct RowView {
    const int64_t *ptr;
    const int32_t *idx;
    const double *val;
    const int64_t *perm;   // null: values in entry order
    int64_t n, nnz;        // rows (= columns) and entries: the bounds checked builds test
};

RowView rows_of(const CsrPat &p, const double *val);   // A
RowView cols_of(const CsrPat &p, const double *val);   // A^T

__device__ __forceinline__ double rv_val(const RowView &v, int64_t e) {
    if (!AIRGA_CK(e, 0, v.nnz, 301)) return 0.0;
    if (!v.perm) return __ldg(v.val + e);
    const int64_t f = __ldg(v.perm + e);
    return AIRGA_CK(f, 0, v.nnz, 302) ? __ldg(v.val + f) : 0.0;
}

// column of entry k, or -1 (checked builds, out of range: recorded)
__device__ __forceinline__ int64_t rv_col(const RowView &v, int64_t k) {
    const int64_t c = __ldg(v.idx + k);
    return AIRGA_CK(c, 0, v.n, 303) ? c : -1;
}

// entry range of row i; checked builds record a row or pointer out of range
// and give an empty range
__device__ __forceinline__ void rv_range(const RowView &v, int64_t i, int64_t &b, int64_t &e) {
    b = e = 0;
    if (!AIRGA_CK(i, 0, v.n, 304)) return;
    b = __ldg(v.ptr + i);
    e = __ldg(v.ptr + i + 1);
    if (!AIRGA_CK(b, 0, v.nnz + 1, 305) || !AIRGA_CK(e, b, v.nnz + 1, 305)) b = e = 0;
}

// (A x)_i, entries summed in stored (column) order
__device__ __forceinline__ double rv_dot(const RowView &v, int64_t i, const double *x) {
    double acc = 0.0;
    int64_t b, e;
    rv_range(v, i, b, e);
    for (int64_t k = b; k < e; ++k) {
        const int64_t c = rv_col(v, k);
        if (c >= 0) acc = fma(rv_val(v, k), x[c], acc);
    }
    return acc;
}

// the same with x read around L1 (x is written by other CTAs of a persistent
// kernel between grid barriers)
__device__ __forceinline__ double rv_dot_cg(const RowView &v, int64_t i, const double *x) {
    double acc = 0.0;
    int64_t b, e;
    rv_range(v, i, b, e);
    for (int64_t k = b; k < e; ++k) {
        const int64_t c = rv_col(v, k);
        if (c >= 0) acc = fma(rv_val(v, k), __ldcg(x + c), acc);
    }
    return acc;
}

}  // namespace airga
