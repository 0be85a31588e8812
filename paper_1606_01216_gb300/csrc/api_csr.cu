// Host side of the C ABI for matrices in general sparse (CSR) storage:
// import, shifted assembly on union patterns, SPAI and SPAI update on a
// general pattern (Eq. 3.1 with S an input; Sec. 3.2), chain application and
// CG.  Band-stored operands meeting a CSR operand are viewed as CSR on the
// full band pattern |i - j| <= 3 (one pattern per size and device, shared).
// No compute happens here.
#include <cstring>
#include <mutex>
#include <tuple>

#include "csr_common.cuh"

namespace airga {

int pcg_csr_grid(int64_t n, int device, int *grid);
size_t pcg_csr_workspace_doubles(int64_t n, int grid);
int launch_pcg_csr(int64_t n, int grid, const RowView &A, int nf, const RowView *fwd,
                   const RowView *tr, const RowView *sym, int symmetrize, const double *F,
                   int32_t m, double *X, double *res_hist, int32_t maxit, double tol, int warm,
                   long long timeout_ns, int fault, int32_t *iters, int32_t *status,
                   double *relres, double *ws, cudaStream_t s);
cudaError_t launch_csr_validate(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                                int32_t *flag, cudaStream_t s);

bool is_csr(airga_mat A) { return A && !A->band && A->csr; }

// ---------------------------------------------------------------------------
// views
// ---------------------------------------------------------------------------

static std::mutex g_band_pat_mu;
static std::vector<std::tuple<int, int64_t, std::weak_ptr<CsrPat>>> g_band_pats;

// The full band pattern of an n x n matrix on the current device, shared.
static int shared_band_pattern(int64_t n, cudaStream_t s, CsrPatPtr *out) {
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_band_pat_mu);
    for (auto &t : g_band_pats) {
        if (std::get<0>(t) == dev && std::get<1>(t) == n) {
            if (auto p = std::get<2>(t).lock()) {
                *out = p;
                return AIRGA_OK;
            }
        }
    }
    CsrPatPtr p;
    int st = band_pattern(n, s, &p);
    if (st) return st;
    bool placed = false;
    for (auto &t : g_band_pats)
        if (std::get<2>(t).expired()) {
            t = std::make_tuple(dev, n, std::weak_ptr<CsrPat>(p));
            placed = true;
            break;
        }
    if (!placed) g_band_pats.emplace_back(dev, n, p);
    *out = p;
    return AIRGA_OK;
}

// CSR pattern and values of a matrix.  A band matrix takes part in the
// general kernels with the pattern of its nonzero entries (a lumped, i.e.
// diagonal, mass matrix stays diagonal); the view is made once and kept with
// the handle, the band staying its primary storage.
int csr_view(airga_mat A, cudaStream_t s, CsrPatPtr *pat, const double **val) {
    if (!A->csr) {
        CsrPatPtr p;
        std::shared_ptr<void> v;
        int st = band_nonzero_csr(A->n, A->band->d, s, &p, &v);
        if (st) return st;
        A->csr = p;
        A->cval = v;
    }
    *pat = A->csr;
    *val = (const double *)A->cval.get();
    return AIRGA_OK;
}

// a band factor for the general kernels: its nonzero entries
static int band_factor_csr(const BandPtr &b, cudaStream_t s, CsrFactor *out) {
    return band_nonzero_csr(b->n, b->d, s, &out->pat, &out->val);
}

// a band array as CSR on the full band pattern (exports keep the storage's
// entries, explicit zeros included)
static int band_export(const BandPtr &b, int64_t n, const double *d, cudaStream_t s,
                       CsrFactor *out) {
    (void)b;
    CsrPatPtr p;
    int st = shared_band_pattern(n, s, &p);
    if (st) return st;
    std::shared_ptr<void> v;
    st = make_buf(sizeof(double) * (size_t)(p->nnz + 1), s, &v);
    if (st) return st;
    AIRGA_CUDA(launch_band_values(*p, d, (double *)v.get(), s));
    out->pat = p;
    out->val = v;
    return AIRGA_OK;
}

// The chain of a preconditioner as CSR factors (band factors converted).
static int chain_csr(airga_precond P, cudaStream_t s, std::vector<CsrFactor> *out) {
    out->clear();
    if (!P->factors.empty()) {
        for (auto &b : P->factors) {
            CsrFactor f;
            int st = band_factor_csr(b, s, &f);
            if (st) return st;
            out->push_back(f);
        }
        return AIRGA_OK;
    }
    *out = P->cfactors;
    return AIRGA_OK;
}

// Union of the patterns X and Y (Y read transposed when y_t), cached on X.
static int union_pattern(const CsrPatPtr &X, const CsrPatPtr &Y, bool y_t, cudaStream_t s,
                         CsrPatPtr *out) {
    if (X.get() == Y.get() && (!y_t || X->symmetric)) {
        *out = X;
        return AIRGA_OK;
    }
    for (auto &u : X->unions)
        if (u.other_transposed == y_t)
            if (auto o = u.other.lock())
                if (o.get() == Y.get()) {
                    *out = u.result;
                    return AIRGA_OK;
                }
    const RowView xv = rows_of(*X, nullptr);
    const RowView yv = y_t ? cols_of(*Y, nullptr) : rows_of(*Y, nullptr);
    CsrPatPtr z;
    int st = csr_union(X->n, xv, yv, s, &z);
    if (st) return st;
    CsrPat::Union u;
    u.other = Y;
    u.other_transposed = y_t;
    u.result = z;
    X->unions.push_back(u);
    *out = z;
    return AIRGA_OK;
}

// ---------------------------------------------------------------------------
// import and assembly
// ---------------------------------------------------------------------------

// flag bits: 1 an entry with |col - row| > 3, 2 malformed (rowptr[0] != 0,
// rowptr[n] != nnz, a decreasing rowptr or a column outside [0, n)).
int csr_check(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
              cudaStream_t s, int32_t *hflag) {
    void *flag = nullptr;
    int st = dev_alloc(&flag, sizeof(int32_t), s);
    if (st) return st;
    *hflag = 0;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_csr_validate(n, nnz, rowptr, col, (int32_t *)flag, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(flag, s);
    if (e != cudaSuccess) return cuda_fail(e, "csr check");
    return AIRGA_OK;
}

int mat_from_csr_general(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                         const double *val, cudaStream_t s, airga_mat *out) {
    CsrPatPtr p;
    std::shared_ptr<void> v;
    int st = csr_import(n, nnz, rowptr, col, val, s, &p, &v);
    if (st) return st;
    auto *m = new airga_mat_s;
    m->n = n;
    m->csr = p;
    m->cval = v;
    *out = m;
    return AIRGA_OK;
}

int assemble_general(airga_mat M, airga_mat K, double alpha, double beta, double sh,
                     cudaStream_t s, airga_mat *A_out) {
    CsrPatPtr pm, pk, pz;
    const double *vm = nullptr, *vk = nullptr;
    int st = csr_view(M, s, &pm, &vm);
    if (!st) st = csr_view(K, s, &pk, &vk);
    if (!st) st = union_pattern(pm, pk, false, s, &pz);
    if (st) return st;
    std::shared_ptr<void> v;
    st = make_buf(sizeof(double) * (size_t)(pz->nnz + 1), s, &v);
    if (st) return st;
    // s^2 M + s (alpha M + beta K) + K = (s^2 + alpha s) M + (1 + beta s) K
    const double cm = sh * sh + alpha * sh, ck = 1.0 + beta * sh;
    AIRGA_CUDA(launch_csr_add(*pz, cm, rows_of(*pm, vm), ck, rows_of(*pk, vk), (double *)v.get(), s));
    auto *m = new airga_mat_s;
    m->n = M->n;
    m->csr = pz;
    m->cval = v;
    *A_out = m;
    return AIRGA_OK;
}

int spmv_general(airga_mat A, const double *X, double *Y, int32_t m, cudaStream_t s) {
    CsrPatPtr p;
    const double *v = nullptr;
    int st = csr_view(A, s, &p, &v);
    if (st) return st;
    AIRGA_CUDA(launch_csr_spmv(A->n, rows_of(*p, v), X, Y, m, s));
    return AIRGA_OK;
}

int true_residual_general(airga_mat A, const double *X, const double *F, int32_t m,
                          double *relres, cudaStream_t s) {
    CsrPatPtr p;
    const double *v = nullptr;
    int st = csr_view(A, s, &p, &v);
    if (st) return st;
    const int nblk = csr_blocks(A->n);
    void *tmp = nullptr;
    st = dev_alloc(&tmp, sizeof(double) * 2 * (size_t)nblk * m, s);
    if (st) return st;
    cudaError_t e = launch_csr_true_residual(A->n, rows_of(*p, v), X, F, m, relres, (double *)tmp,
                                             nblk, s);
    dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "csr true residual");
    return AIRGA_OK;
}

// ---------------------------------------------------------------------------
// SPAI / update on a general pattern
// ---------------------------------------------------------------------------

// One factor: b_j = e_j (A_old null) or A_old e_j; pattern S (null = A's).
// Fills out->col_steps, col_res, rank_flag and *F.
int spai_general(airga_mat A, airga_mat A_old, airga_mat pattern, const airga_options &o,
                 cudaStream_t s, airga_precond_s *out, CsrFactor *F) {
    CsrPatPtr pa, ps;
    const double *va = nullptr, *vold = nullptr;
    int st = csr_view(A, s, &pa, &va);
    if (st) return st;
    if (A_old) {
        CsrPatPtr po;
        st = csr_view(A_old, s, &po, &vold);
        if (st) return st;
        bool same = po.get() == pa.get();
        if (!same) {
            st = csr_same_structure(*po, *pa, s, &same);
            if (st) return st;
        }
        if (!same)
            return fail(AIRGA_E_SHAPE, "spai_update: A_prev and A_next must share one sparsity pattern");
    }
    if (pattern) {
        const double *vp = nullptr;
        st = csr_view(pattern, s, &ps, &vp);
        if (st) return st;
    } else {
        ps = pa;
    }
    const CsrPat::Rows *rows = nullptr;
    st = csr_spai_rows(pa, ps, s, &rows);
    if (st) return st;
    const int64_t n = A->n;
    std::shared_ptr<void> fv;
    st = make_buf(sizeof(double) * (size_t)(ps->nnz + 1), s, &fv);
    if (!st) st = make_buf(sizeof(int32_t) * (size_t)n, s, &out->col_steps);
    if (!st) st = make_buf(sizeof(double) * (size_t)n, s, &out->col_res);
    if (!st) st = make_buf(sizeof(int32_t), s, &out->rank_flag);
    if (st) return st;
    AIRGA_CUDA(cudaMemsetAsync(out->rank_flag.get(), 0, sizeof(int32_t), s));
    AIRGA_CUDA(cudaMemsetAsync(fv.get(), 0, sizeof(double) * (size_t)(ps->nnz + 1), s));
    const bool mr = o.spai_mode == AIRGA_SPAI_MR;
    void *tmp = nullptr;
    double *alpha = nullptr;
    cudaError_t e = cudaSuccess;
    if (mr) {
        const int nblk = csr_blocks(n);
        st = dev_alloc(&tmp, sizeof(double) * (size_t)(2 * nblk + 4), s);
        if (st) return st;
        double *partial = (double *)tmp;
        alpha = partial + 2 * nblk;
        e = launch_csr_mr_alpha(*pa, va, vold, partial, nblk, alpha, s);
    }
    if (e == cudaSuccess)
        e = launch_spai_csr(*pa, va, vold, *ps, *rows, mr ? 1 : 0, mr ? alpha + 2 : nullptr,
                            o.mr_tol, o.mr_relative ? 1 : 0, o.mr_kmax, (double *)fv.get(),
                            (int32_t *)out->col_steps.get(), (double *)out->col_res.get(),
                            (int32_t *)out->rank_flag.get(), s);
    if (tmp) dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "spai (general pattern)");
    F->pat = ps;
    F->val = fv;
    return AIRGA_OK;
}

// 1/2 (F + F^T) on the union of F's pattern and its transpose; entry by
// entry fma(1/2, F(i,j), 1/2 F(j,i)), so the result is exactly symmetric.
int csr_symmetric_part(const CsrFactor &F, cudaStream_t s, CsrFactor *out) {
    CsrPatPtr pz;
    int st = union_pattern(F.pat, F.pat, true, s, &pz);
    if (st) return st;
    std::shared_ptr<void> v;
    st = make_buf(sizeof(double) * (size_t)(pz->nnz + 1), s, &v);
    if (st) return st;
    AIRGA_CUDA(launch_csr_add(*pz, 0.5, rows_of(*F.pat, F.v()), 0.5, cols_of(*F.pat, F.v()),
                              (double *)v.get(), s));
    out->pat = pz;
    out->val = v;
    return AIRGA_OK;
}

int spai_update_general(airga_precond P_prev, airga_mat A_prev, airga_mat A_next,
                        const airga_options &o, cudaStream_t s, airga_precond_s *P) {
    std::vector<CsrFactor> chain;
    int st = chain_csr(P_prev, s, &chain);
    if (st) return st;
    CsrFactor Q;
    st = spai_general(A_next, A_prev, nullptr, o, s, P, &Q);
    if (st) return st;
    chain.push_back(Q);
    P->cfactors = chain;
    return AIRGA_OK;
}

// ---------------------------------------------------------------------------
// chain application and CG
// ---------------------------------------------------------------------------

int precond_apply_general(airga_precond P, const double *r, double *z, int symmetrize,
                          cudaStream_t s) {
    const int64_t n = P->n;
    if (P->cfactors.size() == 1 && symmetrize && P->csym.pat) {
        AIRGA_CUDA(launch_csr_spmv(n, rows_of(*P->csym.pat, P->csym.v()), r, z, 1, s));
        return AIRGA_OK;
    }
    void *tmp = nullptr;
    int st = dev_alloc(&tmp, sizeof(double) * 3 * (size_t)n, s);
    if (st) return st;
    double *t1 = (double *)tmp, *t2 = t1 + n, *t3 = t2 + n;
    cudaError_t e = cudaSuccess;
    const auto &ch = P->cfactors;
    const double *src = r;
    for (size_t f = 0; f < ch.size() && e == cudaSuccess; ++f) {
        double *dst = (f & 1) ? t2 : t1;
        e = launch_csr_spmv(n, rows_of(*ch[f].pat, ch[f].v()), src, dst, 1, s);
        src = dst;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (symmetrize && e == cudaSuccess) {
        src = r;
        size_t cnt = 0;
        for (size_t q = ch.size(); q-- > 0 && e == cudaSuccess; ++cnt) {
            double *dst = (cnt & 1) ? t3 : t1;
            e = launch_csr_spmv(n, cols_of(*ch[q].pat, ch[q].v()), src, dst, 1, s);
            src = dst;
        }
        if (e == cudaSuccess) e = launch_axpby(n, 0.5, src, 0.5, z, s);
    }
    dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "precond apply (general)");
    return AIRGA_OK;
}

int pcg_general(airga_mat A, airga_precond P, const double *F, int32_t m, const airga_options &o,
                double *X, double *res_hist, int32_t *iters, int32_t *status, double *relres,
                int fault, cudaStream_t s) {
    CsrPatPtr pa;
    const double *va = nullptr;
    int st = csr_view(A, s, &pa, &va);
    if (st) return st;
    std::vector<CsrFactor> chain;
    CsrFactor sym;
    bool use_sym = false;
    if (P) {
        st = chain_csr(P, s, &chain);
        if (st) return st;
        if (chain.size() == 1 && o.symmetrize) {
            if (P->csym.pat) {
                sym = P->csym;
            } else {
                st = csr_symmetric_part(chain[0], s, &sym);
                if (st) return st;
            }
            use_sym = true;
        }
    }
    const int nf = (int)chain.size();
    if (nf > kMaxChain) return fail(AIRGA_E_INVALID_ARG, "chain too long");
    RowView fwd[kMaxChain], tr[kMaxChain], symv;
    for (int k = 0; k < nf; ++k) {
        fwd[k] = rows_of(*chain[k].pat, chain[k].v());
        tr[k] = cols_of(*chain[k].pat, chain[k].v());
    }
    if (use_sym) symv = rows_of(*sym.pat, sym.v());
    int dev = 0, grid = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    st = pcg_csr_grid(A->n, dev, &grid);
    if (st) return st;
    void *ws = nullptr;
    st = dev_alloc(&ws, sizeof(double) * pcg_csr_workspace_doubles(A->n, grid) + 64, s);
    if (st) return st;
    st = launch_pcg_csr(A->n, grid, rows_of(*pa, va), use_sym ? 0 : nf, fwd, tr,
                        use_sym ? &symv : nullptr, o.symmetrize ? 1 : 0, F, m, X, res_hist,
                        o.maxit, o.tol, o.warm_start ? 1 : 0,
                        (long long)o.barrier_timeout_ms * 1000000ll, fault, iters, status, relres,
                        (double *)ws, s);
    dev_free(ws, s);
    return st;
}

static int64_t band_nnz(int64_t n) {
    int64_t nnz = 0;
    for (int64_t d = -kHalf; d <= kHalf; ++d) {
        const int64_t len = n - (d < 0 ? -d : d);
        if (len > 0) nnz += len;
    }
    return nnz;
}

// factor k of a chain for export (band factors on their full band pattern)
static int factor_k(airga_precond P, int32_t k, cudaStream_t s, CsrFactor *out) {
    if (!P->factors.empty()) return band_export(P->factors[k], P->n, P->factors[k]->d, s, out);
    *out = P->cfactors[k];
    return AIRGA_OK;
}

static int copy_csr(const CsrPat &p, const double *v, int64_t *rowptr, int32_t *col, double *val,
                    cudaStream_t s) {
    if (rowptr)
        AIRGA_CUDA(cudaMemcpyAsync(rowptr, p.rowptr, sizeof(int64_t) * (size_t)(p.n + 1),
                                   cudaMemcpyDeviceToDevice, s));
    if (col && p.nnz)
        AIRGA_CUDA(cudaMemcpyAsync(col, p.col, sizeof(int32_t) * (size_t)p.nnz,
                                   cudaMemcpyDeviceToDevice, s));
    if (val && p.nnz)
        AIRGA_CUDA(cudaMemcpyAsync(val, v, sizeof(double) * (size_t)p.nnz, cudaMemcpyDeviceToDevice, s));
    return AIRGA_OK;
}

}  // namespace airga

using namespace airga;

extern "C" {

int airga_mat_is_banded(airga_mat A) { return A && A->band ? 1 : 0; }

int64_t airga_mat_nnz(airga_mat A) {
    if (!A) return 0;
    if (A->band) return band_nnz(A->n);
    return A->csr ? A->csr->nnz : 0;
}

int airga_mat_to_csr(airga_mat A, int64_t *rowptr, int32_t *col, double *val, void *stream) {
    int st = check_any(A, "A");
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (A->band) {
        CsrFactor f;
        st = band_export(A->band, A->n, A->band->d, s, &f);
        if (st) return st;
        return copy_csr(*f.pat, f.v(), rowptr, col, val, s);
    }
    return copy_csr(*A->csr, (const double *)A->cval.get(), rowptr, col, val, s);
}

int64_t airga_precond_factor_nnz(airga_precond P, int32_t k) {
    if (!P || k < 0) return 0;
    if (!P->factors.empty()) return k < (int32_t)P->factors.size() ? band_nnz(P->n) : 0;
    return k < (int32_t)P->cfactors.size() ? P->cfactors[k].pat->nnz : 0;
}

int airga_precond_is_banded(airga_precond P) { return P && !P->factors.empty() ? 1 : 0; }

int airga_precond_factor_csr(airga_precond P, int32_t k, int64_t *rowptr, int32_t *col,
                             double *val, void *stream) {
    if (!P || k < 0 || k >= airga_precond_length(P))
        return fail(AIRGA_E_INVALID_ARG, "bad factor request");
    cudaStream_t s = (cudaStream_t)stream;
    CsrFactor f;
    int st = factor_k(P, k, s, &f);
    if (st) return st;
    return copy_csr(*f.pat, f.v(), rowptr, col, val, s);
}

int airga_precond_from_csr(int64_t n, int32_t nfactors, const int64_t *nnz,
                           const int64_t *const *rowptr, const int32_t *const *col,
                           const double *const *val, void *stream, airga_precond *P_out) {
    if (!P_out) return fail(AIRGA_E_INVALID_ARG, "P_out is NULL");
    *P_out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX || nfactors < 1 || nfactors > kMaxChain || !nnz ||
        !rowptr || !col || !val)
        return fail(AIRGA_E_INVALID_ARG, "bad factor list");
    cudaStream_t s = (cudaStream_t)stream;
    auto *P = new airga_precond_s;
    P->n = n;
    int st = AIRGA_OK;
    for (int32_t k = 0; k < nfactors && !st; ++k) {
        if (nnz[k] < 0 || !rowptr[k] || (nnz[k] > 0 && (!col[k] || !val[k]))) {
            st = fail(AIRGA_E_INVALID_ARG, "bad CSR arrays of a factor");
            break;
        }
        int32_t flag = 0;
        st = csr_check(n, nnz[k], rowptr[k], col[k], s, &flag);
        if (!st && (flag & 2)) st = fail(AIRGA_E_INVALID_ARG, "CSR arrays of a factor malformed");
        CsrFactor f;
        if (!st) st = csr_import(n, nnz[k], rowptr[k], col[k], val[k], s, &f.pat, &f.val);
        if (!st) P->cfactors.push_back(f);
    }
    if (!st && nfactors == 1) st = csr_symmetric_part(P->cfactors[0], s, &P->csym);
    if (st) {
        delete P;
        return st;
    }
    *P_out = P;
    return AIRGA_OK;
}

}  // extern "C"
