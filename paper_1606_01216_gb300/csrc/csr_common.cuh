// Row access to general sparse matrices for the CSR kernels.
//
// A RowView reads row i of a matrix as the entries e in [ptr[i], ptr[i+1])
// with column idx[e] and value val[perm ? perm[e] : e].  The CSR arrays of a
// pattern give the matrix itself; its CSC arrays with the transposition map
// give the transpose (row i of A^T = column i of A) over the same value
// array, so A^T r needs no second copy of the values.
#pragma once

#include "airga_internal.cuh"

namespace airga {

struct RowView {
    const int64_t *ptr;
    const int32_t *idx;
    const double *val;
    const int64_t *perm;   // null: values in entry order
};

RowView rows_of(const CsrPat &p, const double *val);   // A
RowView cols_of(const CsrPat &p, const double *val);   // A^T

__device__ __forceinline__ double rv_val(const RowView &v, int64_t e) {
    return v.perm ? __ldg(v.val + __ldg(v.perm + e)) : __ldg(v.val + e);
}

// (A x)_i, entries summed in stored (column) order
__device__ __forceinline__ double rv_dot(const RowView &v, int64_t i, const double *x) {
    double acc = 0.0;
    const int64_t b = __ldg(v.ptr + i), e = __ldg(v.ptr + i + 1);
    for (int64_t k = b; k < e; ++k) acc = fma(rv_val(v, k), x[__ldg(v.idx + k)], acc);
    return acc;
}

// the same with x read around L1 (x is written by other CTAs of a persistent
// kernel between grid barriers)
__device__ __forceinline__ double rv_dot_cg(const RowView &v, int64_t i, const double *x) {
    double acc = 0.0;
    const int64_t b = __ldg(v.ptr + i), e = __ldg(v.ptr + i + 1);
    for (int64_t k = b; k < e; ++k) acc = fma(rv_val(v, k), __ldcg(x + __ldg(v.idx + k)), acc);
    return acc;
}

}  // namespace airga
