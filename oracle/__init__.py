"""CPU oracle for the shifted-system SPAI/PCG path — TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's cpu_baseline/reference leg use
this package.  The product (the CUDA library and its binding) never imports
it.  All arithmetic lives in airga_oracle.c (plain FP64 C); this module only
marshals numpy arrays through ctypes.

Matrices are scipy-free CSR triples (rowptr int64, col int32, val float64)
with sorted column indices.  Patterns for SPAI are given by columns
(colptr int64, rowidx int32); for a structurally symmetric matrix the CSR
arrays of A serve directly as that pattern.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EARG, EBREAKDOWN, EMAXIT, ERANK, ENOMEM = 0, 1, 3, 4, 6, 8

_libs = {}
_openmp = False


def use_openmp(flag: bool) -> None:
    """Route the calls below to the OpenMP build (all host cores) or back to
    the serial parity reference."""
    global _openmp
    _openmp = bool(flag)


def threads() -> int:
    """Threads the selected build uses."""
    return int(lib().ora_threads())


def lib():
    key = "omp" if _openmp else "serial"
    if key not in _libs:
        path = _build.build(openmp=_openmp)
        L = C.CDLL(path)
        L.ora_threads.argtypes = []
        L.ora_threads.restype = C.c_int
        dp, ip64, ip32 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        L.ora_shifted.argtypes = [C.c_int64, dp, dp, C.c_double, C.c_double, C.c_double, dp]
        L.ora_shifted.restype = None
        for f in (L.ora_spmv, L.ora_spmv_t):
            f.argtypes = [C.c_int64, ip64, ip32, dp, dp, dp]
            f.restype = None
        L.ora_lsq_qr.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.ora_lsq_qr.restype = C.c_int
        L.ora_spai.argtypes = [C.c_int64, ip64, ip32, dp, dp, ip64, ip32, dp, dp]
        L.ora_spai.restype = C.c_int
        L.ora_alpha_build.argtypes = [C.c_int64, ip64, ip32, dp]
        L.ora_alpha_build.restype = C.c_double
        L.ora_alpha_update.argtypes = [C.c_int64, ip64, dp, dp]
        L.ora_alpha_update.restype = C.c_double
        L.ora_spai_mr.argtypes = [C.c_int64, ip64, ip32, dp, dp, ip64, ip32, C.c_double,
                                  C.c_double, C.c_int, C.c_int, dp, ip32, dp]
        L.ora_spai_mr.restype = C.c_int
        L.ora_pcg.argtypes = [C.c_int64, ip64, ip32, dp, C.c_int, C.POINTER(ip64),
                              C.POINTER(ip32), C.POINTER(dp), C.c_int, dp, C.c_double, C.c_int,
                              dp, dp, ip32]
        L.ora_pcg.restype = C.c_int
        L.ora_chol_solve.argtypes = [C.c_int64, ip64, ip32, dp, C.c_int, dp, dp]
        L.ora_chol_solve.restype = C.c_int
        _libs[key] = L
    return _libs[key]


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _i64(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class CSR:
    """Plain CSR triple."""

    def __init__(self, n, rowptr, col, val):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)

    def dense(self):
        A = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        A[rows, self.col] = self.val
        return A

    def transpose(self):
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr)).astype(np.int64)
        order = np.lexsort((rows, self.col))
        rp = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(np.bincount(self.col, minlength=self.n), out=rp[1:])
        return CSR(self.n, rp, rows[order], self.val[order])


def dense_to_csr(A, pattern=None):
    """Dense -> CSR, on the given CSR pattern's transpose-closed support if
    provided (keeps explicit zeros), else on the nonzeros."""
    n = A.shape[0]
    if pattern is None:
        mask = A != 0
    else:
        mask = np.zeros((n, n), dtype=bool)
        rows = np.repeat(np.arange(n), np.diff(pattern.rowptr))
        mask[rows, pattern.col] = True
        mask |= mask.T
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(1), out=rp[1:])
    r, c = np.nonzero(mask)
    return CSR(n, rp, c.astype(np.int32), A[r, c])


# ---------------------------------------------------------------------------

def shifted(m_val, k_val, alpha, beta, s):
    m_val, k_val = _f64(m_val), _f64(k_val)
    out = np.empty_like(m_val)
    lib().ora_shifted(m_val.size, _d(m_val), _d(k_val), alpha, beta, s, _d(out))
    return out


def spmv(A: CSR, x):
    x = _f64(x)
    y = np.empty(A.n)
    lib().ora_spmv(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val), _d(x), _d(y))
    return y


def spmv_t(A: CSR, x):
    x = _f64(x)
    y = np.empty(A.n)
    lib().ora_spmv_t(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val), _d(x), _d(y))
    return y


def lsq_qr(Ahat, b):
    """Dense LS min ||b - Ahat x|| by the oracle's Householder QR."""
    Ahat = np.array(Ahat, dtype=np.float64, order="F")
    b = np.array(b, dtype=np.float64)
    rows, cols = Ahat.shape
    x = np.empty(cols)
    st = lib().ora_lsq_qr(rows, cols, _d(Ahat), _d(b), _d(x))
    return x, st


def spai(A: CSR, pattern: CSR | None = None, A_old: CSR | None = None, want_colres=False):
    """Exact fixed-pattern SPAI (A_old None) or SPAI-update factor Q.

    pattern: CSR whose *columns* give J_j (a symmetric pattern's CSR works
    as is); defaults to A's pattern.  Returns the factor as CSR (rows), plus
    per-column residuals when asked."""
    pat = pattern if pattern is not None else A
    pcp, pcr = pat.rowptr, pat.col          # read as columns of the pattern
    pval = np.zeros(pcr.size)
    colres = np.empty(A.n) if want_colres else None
    if A_old is not None and (A_old.rowptr.size != A.rowptr.size or
                              not np.array_equal(A_old.col, A.col)):
        raise ValueError("A_old must share A's CSR pattern")
    st = lib().ora_spai(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val),
                        _d(A_old.val) if A_old is not None else None,
                        _i64(pcp), _i32(pcr), _d(pval), _d(colres))
    if st != OK:
        raise RuntimeError("ora_spai status %d" % st)
    # pval is laid out by columns: (colptr=pcp, rowidx=pcr) -> CSR of factor^T
    FT = CSR(A.n, pcp, pcr, pval)
    F = FT.transpose()
    return (F, colres) if want_colres else F


def alpha_build(A: CSR):
    return lib().ora_alpha_build(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val))


def alpha_update(A_old: CSR, A_new: CSR):
    return lib().ora_alpha_update(A_new.n, _i64(A_new.rowptr), _d(A_old.val), _d(A_new.val))


def spai_mr(A: CSR, tol=0.01, kmax=50, pattern: CSR | None = None, A_old: CSR | None = None,
            relative: bool = False):
    """The paper's MR iteration (Algorithm 2, or Algorithm 4 when A_old is
    given).  A column stops when ||r|| <= tol (the paper's test), or with
    relative=True when ||r|| <= tol ||b_j||.  Returns (factor CSR, steps per
    column, final column residuals, alpha0)."""
    pat = pattern if pattern is not None else A
    alpha0 = alpha_build(A) if A_old is None else alpha_update(A_old, A)
    pval = np.zeros(pat.col.size)
    steps = np.zeros(A.n, dtype=np.int32)
    colres = np.empty(A.n)
    st = lib().ora_spai_mr(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val),
                           _d(A_old.val) if A_old is not None else None,
                           _i64(pat.rowptr), _i32(pat.col), alpha0, tol,
                           1 if relative else 0, kmax,
                           _d(pval), _i32(steps), _d(colres))
    if st != OK:
        raise RuntimeError("ora_spai_mr status %d" % st)
    F = CSR(A.n, pat.rowptr, pat.col, pval).transpose()
    return F, steps, colres, alpha0


def pcg(A: CSR, b, factors=(), symmetrize=True, tol=1e-10, maxit=10000, x0=None):
    """PCG with z = 1/2 (C + C^T) r, C = factors[-1] ... factors[0].
    Returns (x, iters, status, history)."""
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    hist = np.full(maxit + 1, np.nan)
    it = np.zeros(1, dtype=np.int32)
    nf = len(factors)
    RP = (C.POINTER(C.c_int64) * max(nf, 1))(*[_i64(f.rowptr) for f in factors])
    CI = (C.POINTER(C.c_int32) * max(nf, 1))(*[_i32(f.col) for f in factors])
    VV = (C.POINTER(C.c_double) * max(nf, 1))(*[_d(f.val) for f in factors])
    st = lib().ora_pcg(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val), nf, RP, CI, VV,
                       1 if symmetrize else 0, _d(b), tol, maxit, _d(x), _d(hist), _i32(it))
    k = int(it[0])
    return x, k, st, hist[:k + 1]


def chol_solve(A: CSR, B):
    B = np.asfortranarray(np.atleast_2d(np.asarray(B, dtype=np.float64).T).T)
    if B.ndim == 1:
        B = B[:, None]
    X = np.empty_like(B, order="F")
    st = lib().ora_chol_solve(A.n, _i64(A.rowptr), _i32(A.col), _d(A.val), B.shape[1],
                              _d(B), _d(X))
    if st != OK:
        raise RuntimeError("ora_chol_solve status %d" % st)
    return X


def from_beam(beam, which: str):
    """CSR of M ('m') or K ('k') from a workloads.BeamCSR."""
    return CSR(beam.n, beam.rowptr, beam.col, beam.m_val if which == "m" else beam.k_val)


def shifted_csr(beam, alpha, beta, s):
    """A(s) = s^2 M + s D + K on the beam's pattern, as CSR."""
    return CSR(beam.n, beam.rowptr, beam.col, shifted(beam.m_val, beam.k_val, alpha, beta, s))
