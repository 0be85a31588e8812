// Host side of the C ABI declared in include/airga.h: argument checks,
// handle lifetime, the library's stream-ordered memory pool and kernel
// launch sequencing.  No compute happens here.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "airga_internal.cuh"

namespace airga {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? AIRGA_E_OOM : AIRGA_E_CUDA;
}

// ---------------------------------------------------------------------------
// one stream-ordered pool per device (memory is kept for reuse until trim)
// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;

static int pool_for_current(cudaMemPool_t *out) {
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if ((int)g_pools.size() <= dev) g_pools.resize(dev + 1, nullptr);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        AIRGA_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = ~0ull;
        AIRGA_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return AIRGA_OK;
}

int dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (take_fault(AIRGA_FAULT_ALLOC))
        return fail(AIRGA_E_OOM, "device allocation: injected failure (AIRGA_FAULT_ALLOC)");
    cudaMemPool_t pool = nullptr;
    int st = pool_for_current(&pool);
    if (st) return st;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "device allocation");
    }
    return AIRGA_OK;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

Band::~Band() {
    if (d) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != device) cudaSetDevice(device);
        cudaFreeAsync(d, stream);
        if (cur != device) cudaSetDevice(cur);
    }
}

int make_band(int64_t n, cudaStream_t s, BandPtr *out) {
    auto b = std::make_shared<Band>();
    b->n = n;
    b->stream = s;
    cudaGetDevice(&b->device);
    void *p = nullptr;
    int st = dev_alloc(&p, sizeof(double) * (size_t)kBand * (size_t)n, s);
    if (st) return st;
    b->d = (double *)p;
    *out = b;
    return AIRGA_OK;
}

// shared_ptr<void> owning a pool allocation
int make_buf(size_t bytes, cudaStream_t s, std::shared_ptr<void> *out) {
    void *p = nullptr;
    int st = dev_alloc(&p, bytes, s);
    if (st) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    *out = std::shared_ptr<void>(p, [s, dev](void *q) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != dev) cudaSetDevice(dev);
        cudaFreeAsync(q, s);
        if (cur != dev) cudaSetDevice(cur);
    });
    return AIRGA_OK;
}

static cudaStream_t S(void *stream) { return (cudaStream_t)stream; }

// device flag of the beam zero structure, detected from the band on the stream
static int detect_flag(airga_mat_s *m, cudaStream_t s) {
    int st = make_buf(sizeof(int32_t), s, &m->pairz);
    if (st) return st;
    AIRGA_CUDA(cudaMemsetAsync(m->pairz.get(), 1, sizeof(int32_t), s));
    AIRGA_CUDA(launch_detect_pairz(m->n, m->band->d, (int32_t *)m->pairz.get(), s));
    return AIRGA_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static std::atomic<int> g_fault{AIRGA_FAULT_NONE};

bool take_fault(int kind) {
    int expected = kind;
    return g_fault.compare_exchange_strong(expected, AIRGA_FAULT_NONE);
}

cudaError_t injected_launch_error() {
    return take_fault(AIRGA_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources : cudaSuccess;
}

static std::atomic<int> g_forced_kind{0};

int forced_pcg_kind() { return g_forced_kind.load(); }
static std::atomic<int32_t *> g_place{nullptr};
int32_t *placement_buffer() { return g_place.load(); }

static_assert(sizeof(airga_options) == 72, "airga_options layout (the Python binding mirrors it)");

int check_options(const airga_options *o) {
    if (!(o->tol >= 0.0) || !std::isfinite(o->tol)) return fail(AIRGA_E_INVALID_ARG, "tol must be finite and >= 0");
    if (o->maxit < 0) return fail(AIRGA_E_INVALID_ARG, "maxit must be >= 0");
    if (o->spai_mode != AIRGA_SPAI_QR && o->spai_mode != AIRGA_SPAI_MR &&
        o->spai_mode != AIRGA_SPAI_NE)
        return fail(AIRGA_E_INVALID_ARG, "spai_mode must be AIRGA_SPAI_QR, AIRGA_SPAI_MR or AIRGA_SPAI_NE");
    if (!(o->mr_tol >= 0.0)) return fail(AIRGA_E_INVALID_ARG, "mr_tol must be >= 0");
    if (o->mr_kmax < 0) return fail(AIRGA_E_INVALID_ARG, "mr_kmax must be >= 0");
    if (o->pattern_hbw < 0 || o->pattern_hbw > 3)
        return fail(AIRGA_E_INVALID_ARG, "pattern_hbw must be in 0..3");
    if (o->barrier_timeout_ms <= 0) return fail(AIRGA_E_INVALID_ARG, "barrier_timeout_ms must be > 0");
    if (o->sm_share < 1 || o->sm_share > 3) return fail(AIRGA_E_INVALID_ARG, "sm_share must be 1, 2 or 3");
    if (!(o->inner_tol > 0.0) || !(o->inner_tol < 1.0))
        return fail(AIRGA_E_INVALID_ARG, "inner_tol must be in (0, 1)");
    if (o->max_outer < 1) return fail(AIRGA_E_INVALID_ARG, "max_outer must be >= 1");
    return AIRGA_OK;
}

// a matrix in either storage
int check_any(airga_mat A, const char *name) {
    if (!A || (!A->band && !A->csr) || A->n < 1)
        return fail(AIRGA_E_INVALID_ARG, std::string(name) + " is not a valid matrix");
    return AIRGA_OK;
}

// a band-7 matrix (calls with no general sparse form)
int check_mat(airga_mat A, const char *name) {
    int st = check_any(A, name);
    if (st) return st;
    if (!A->band)
        return fail(AIRGA_E_UNSUPPORTED, std::string(name) +
                                             " is stored as a general sparse (CSR) matrix; this "
                                             "call needs band-7 storage");
    return AIRGA_OK;
}

// Build one SPAI / SPAI-update factor of A (b_j = e_j, or A_old e_j) into a
// new band; per-column results into `out`'s status buffers.
static int spai_factor(airga_mat A, airga_mat A_old, const airga_options &o, cudaStream_t s,
                       airga_precond_s *out, BandPtr *F) {
    const int64_t n = A->n;
    int st = make_band(n, s, F);
    if (st) return st;
    st = make_buf(sizeof(int32_t) * (size_t)n, s, &out->col_steps);
    if (st) return st;
    st = make_buf(sizeof(double) * (size_t)n, s, &out->col_res);
    if (st) return st;
    st = make_buf(sizeof(int32_t), s, &out->rank_flag);
    if (st) return st;
    AIRGA_CUDA(cudaMemsetAsync(out->rank_flag.get(), 0, sizeof(int32_t), s));
    const double *Aold = A_old ? A_old->band->d : nullptr;
    if (o.spai_mode == AIRGA_SPAI_NE && o.pattern_hbw == 3) {
        AIRGA_CUDA(cudaMemsetAsync(out->col_steps.get(), 0, sizeof(int32_t) * (size_t)n, s));
        void *tmp = nullptr;
        st = dev_alloc(&tmp, sizeof(double) * 7 * (size_t)n + sizeof(int32_t) * (size_t)(n + 2), s);
        if (st) return st;
        double *U = (double *)tmp;
        int32_t *fb = (int32_t *)(U + 7 * (size_t)n);
        const cudaError_t e = launch_spai_ne(n, A->band->d, Aold, (*F)->d, (double *)out->col_res.get(),
                                             o.want_colres != 0, (int32_t *)out->rank_flag.get(),
                                             (int32_t *)out->col_steps.get(), U, fb,
                                             (const int32_t *)A->pairz.get(), s);
        dev_free(tmp, s);
        if (e != cudaSuccess) return cuda_fail(e, "spai NE launch");
        return AIRGA_OK;
    }
    if (o.spai_mode == AIRGA_SPAI_QR || o.spai_mode == AIRGA_SPAI_NE) {
        AIRGA_CUDA(cudaMemsetAsync(out->col_steps.get(), 0, sizeof(int32_t) * (size_t)n, s));
        AIRGA_CUDA(launch_spai_qr(n, o.pattern_hbw, A->band->d, Aold, (*F)->d,
                                  (double *)out->col_res.get(), (int32_t *)out->rank_flag.get(),
                                  (const int32_t *)A->pairz.get(),
                                  A_old ? (const int32_t *)A_old->pairz.get() : nullptr, s));
        return AIRGA_OK;
    }
    const int nblk = mr_alpha_blocks(n);
    void *tmp = nullptr;
    st = dev_alloc(&tmp, sizeof(double) * (size_t)(2 * nblk + 4), s);
    if (st) return st;
    double *partial = (double *)tmp, *alpha = partial + 2 * nblk;
    cudaError_t e = launch_mr_alpha(n, A->band->d, Aold, partial, nblk, alpha, s);
    if (e == cudaSuccess)
        e = launch_spai_mr(n, o.pattern_hbw, A->band->d, Aold, alpha + 2, o.mr_tol,
                           o.mr_relative ? 1 : 0, o.mr_kmax,
                           (*F)->d, (int32_t *)out->col_steps.get(), (double *)out->col_res.get(), s);
    dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "spai MR launch");
    return AIRGA_OK;
}

}  // namespace airga

using namespace airga;

extern "C" {

void airga_options_default(airga_options *o) {
    if (!o) return;
    o->tol = 1e-10;
    o->maxit = 20000;
    o->spai_mode = AIRGA_SPAI_QR;
    o->mr_tol = 0.01;
    o->mr_kmax = 50;
    o->symmetrize = 1;
    o->pattern_hbw = 3;
    o->warm_start = 0;
    o->barrier_timeout_ms = 2000;
    o->want_colres = 1;
    o->sm_share = 1;
    o->reserved0 = 0;
    o->inner_tol = 3e-4;   // fewest FP32 + FP64 iterations on the beam workloads (measured)
    o->max_outer = 12;
    o->mr_relative = 0;    // the paper's ||r|| <= tol
}

const char *airga_status_string(int s) {
    switch (s) {
        case AIRGA_OK: return "ok";
        case AIRGA_E_INVALID_ARG: return "invalid argument";
        case AIRGA_E_SHAPE: return "shape mismatch";
        case AIRGA_E_BREAKDOWN: return "CG breakdown (not SPD, or (r,z) zero / not finite)";
        case AIRGA_E_MAXIT: return "iteration cap reached";
        case AIRGA_E_TIMEOUT: return "grid barrier timed out";
        case AIRGA_E_RANK: return "rank-deficient least-squares block";
        case AIRGA_E_CUDA: return "CUDA error";
        case AIRGA_E_OOM: return "out of device memory";
        case AIRGA_E_UNSUPPORTED: return "operation not available for this matrix storage";
        default: return "unknown status";
    }
}

const char *airga_last_error(void) { return g_last_error.c_str(); }

int airga_version(void) { return 100; }

// ---------------------------------------------------------------------------
// matrices
// ---------------------------------------------------------------------------
int airga_mat_from_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                       const double *val, void *stream, airga_mat *out) {
    TraceScope trace_("airga_mat_from_csr", stream);
    if (!out) return fail(AIRGA_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(AIRGA_E_INVALID_ARG, "n must be in [1, 2^31)");
    if (nnz < 0 || nnz > (int64_t)INT32_MAX * 64 || !rowptr || (nnz > 0 && (!col || !val)))
        return fail(AIRGA_E_INVALID_ARG, "bad CSR arrays");
    cudaStream_t s = S(stream);
    int32_t hflag = 0;
    int st = csr_check(n, nnz, rowptr, col, s, &hflag);
    if (st) return st;
    if (hflag & 2)
        return fail(AIRGA_E_INVALID_ARG,
                    "CSR arrays malformed (rowptr[0] != 0, rowptr[n] != nnz, decreasing rowptr "
                    "or a column index outside [0, n))");
    if (hflag & 1) return mat_from_csr_general(n, nnz, rowptr, col, val, s, out);
    BandPtr b;
    st = make_band(n, s, &b);
    if (st) return st;
    void *flag = nullptr;
    st = dev_alloc(&flag, sizeof(int32_t), s);
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_csr_to_band(n, rowptr, col, val, b->d, (int32_t *)flag, s);
    dev_free(flag, s);
    if (e != cudaSuccess) return cuda_fail(e, "mat_from_csr");
    auto *m = new airga_mat_s;
    m->n = n;
    m->band = b;
    st = detect_flag(m, s);
    if (st) {
        delete m;
        return st;
    }
    *out = m;
    return AIRGA_OK;
}

int airga_mat_from_band(int64_t n, const double *band, void *stream, airga_mat *out) {
    TraceScope trace_("airga_mat_from_band", stream);
    if (!out) return fail(AIRGA_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX || !band) return fail(AIRGA_E_INVALID_ARG, "bad band input");
    cudaStream_t s = S(stream);
    BandPtr b;
    int st = make_band(n, s, &b);
    if (st) return st;
    AIRGA_CUDA(cudaMemcpyAsync(b->d, band, sizeof(double) * kBand * (size_t)n,
                               cudaMemcpyDeviceToDevice, s));
    auto *m = new airga_mat_s;
    m->n = n;
    m->band = b;
    st = detect_flag(m, s);
    if (st) {
        delete m;
        return st;
    }
    *out = m;
    return AIRGA_OK;
}

int airga_mat_to_band(airga_mat A, double *band, void *stream) {
    int st = check_mat(A, "A");
    if (st) return st;
    if (!band) return fail(AIRGA_E_INVALID_ARG, "band is NULL");
    AIRGA_CUDA(cudaMemcpyAsync(band, A->band->d, sizeof(double) * kBand * (size_t)A->n,
                               cudaMemcpyDeviceToDevice, S(stream)));
    return AIRGA_OK;
}

int64_t airga_mat_rows(airga_mat A) { return A ? A->n : 0; }

void airga_mat_free(airga_mat A) { delete A; }

// ---------------------------------------------------------------------------
// the path
// ---------------------------------------------------------------------------
int airga_assemble_shifted(airga_mat M, airga_mat K, double alpha, double beta, double s,
                           void *stream, airga_mat *A_out) {
    TraceScope trace_("airga_assemble_shifted", stream);
    if (!A_out) return fail(AIRGA_E_INVALID_ARG, "A_out is NULL");
    *A_out = nullptr;
    int st = check_any(M, "M");
    if (!st) st = check_any(K, "K");
    if (st) return st;
    if (M->n != K->n) return fail(AIRGA_E_SHAPE, "M and K differ in size");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(s))
        return fail(AIRGA_E_INVALID_ARG, "alpha, beta and s must be finite");
    cudaStream_t cs = S(stream);
    if (!M->band || !K->band) return assemble_general(M, K, alpha, beta, s, cs, A_out);
    BandPtr b;
    st = make_band(M->n, cs, &b);
    if (st) return st;
    std::shared_ptr<void> flag;
    st = make_buf(sizeof(int32_t), cs, &flag);
    if (st) return st;
    const int32_t *fm = (const int32_t *)(M->pairz ? M->pairz.get() : nullptr);
    const int32_t *fk = (const int32_t *)(K->pairz ? K->pairz.get() : nullptr);
    std::shared_ptr<void> packed;
    if (fm && fk && M->n % 2 == 0) {
        // both inputs may be beams (decided on the device): assemble by row
        // pairs and write the packed beam stencil the CG kernel reads
        st = make_buf(sizeof(double) * 5 * (size_t)M->n, cs, &packed);
        if (st) return st;
        AIRGA_CUDA(launch_assemble_pack(M->n, M->band->d, K->band->d, alpha, beta, s, b->d,
                                        (double *)packed.get(), cs, fm, fk, (int32_t *)flag.get()));
    } else {
        AIRGA_CUDA(launch_assemble(M->n, M->band->d, K->band->d, alpha, beta, s, b->d, cs, fm, fk,
                                   (int32_t *)flag.get()));
    }
    auto *m = new airga_mat_s;
    m->n = M->n;
    m->band = b;
    m->pairz = flag;
    m->packed = packed;
    *A_out = m;
    return AIRGA_OK;
}

int airga_spmv(airga_mat A, const double *X, double *Y, int32_t m, void *stream) {
    TraceScope trace_("airga_spmv", stream);
    int st = check_any(A, "A");
    if (st) return st;
    if (m < 0 || (m > 0 && (!X || !Y))) return fail(AIRGA_E_INVALID_ARG, "bad spmv operands");
    if (m == 0) return AIRGA_OK;
    if (!A->band) return spmv_general(A, X, Y, m, S(stream));
    AIRGA_CUDA(launch_spmv(A->n, A->band->d, X, Y, m, S(stream)));
    return AIRGA_OK;
}

int airga_spai_build(airga_mat A, airga_mat pattern, const airga_options *opt, void *stream,
                     airga_precond *P_out) {
    TraceScope trace_("airga_spai_build", stream);
    if (!P_out) return fail(AIRGA_E_INVALID_ARG, "P_out is NULL");
    *P_out = nullptr;
    int st = check_any(A, "A");
    if (!st && pattern) st = check_any(pattern, "pattern");
    if (st) return st;
    if (pattern && pattern->n != A->n) return fail(AIRGA_E_SHAPE, "pattern and A differ in size");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    st = check_options(&o);
    if (st) return st;
    cudaStream_t s = S(stream);
    auto *P = new airga_precond_s;
    P->n = A->n;
    if (!A->band || (pattern && !pattern->band)) {
        // general pattern: CSR factor and its symmetric part
        CsrFactor F;
        st = spai_general(A, nullptr, pattern, o, s, P, &F);
        if (!st) st = csr_symmetric_part(F, s, &P->csym);
        if (st) {
            delete P;
            return st;
        }
        P->cfactors.push_back(F);
        *P_out = P;
        return AIRGA_OK;
    }
    BandPtr F;
    st = spai_factor(A, nullptr, o, s, P, &F);
    if (!st) st = make_band(A->n, s, &P->psym);
    if (!st) {
        cudaError_t e = launch_symmetrize(A->n, F->d, P->psym->d, s);
        if (e != cudaSuccess) st = cuda_fail(e, "symmetrize");
    }
    if (st) {
        delete P;
        return st;
    }
    P->factors.push_back(F);
    *P_out = P;
    return AIRGA_OK;
}

int airga_spai_update(airga_precond P_prev, airga_mat A_prev, airga_mat A_next,
                      const airga_options *opt, void *stream, airga_precond *P_out) {
    TraceScope trace_("airga_spai_update", stream);
    if (!P_out) return fail(AIRGA_E_INVALID_ARG, "P_out is NULL");
    *P_out = nullptr;
    if (!P_prev || (P_prev->factors.empty() && P_prev->cfactors.empty()))
        return fail(AIRGA_E_INVALID_ARG, "P_prev is not a valid preconditioner");
    int st = check_any(A_prev, "A_prev");
    if (!st) st = check_any(A_next, "A_next");
    if (st) return st;
    if (A_prev->n != A_next->n || P_prev->n != A_next->n)
        return fail(AIRGA_E_SHAPE, "P_prev, A_prev and A_next differ in size");
    if ((int)(P_prev->factors.size() + P_prev->cfactors.size()) + 1 > kMaxChain)
        return fail(AIRGA_E_INVALID_ARG, "preconditioner chain longer than 16 factors");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    st = check_options(&o);
    if (st) return st;
    cudaStream_t s = S(stream);
    auto *P = new airga_precond_s;
    P->n = A_next->n;
    if (P_prev->factors.empty() || !A_prev->band || !A_next->band) {
        st = spai_update_general(P_prev, A_prev, A_next, o, s, P);
        if (st) {
            delete P;
            return st;
        }
        *P_out = P;
        return AIRGA_OK;
    }
    BandPtr Q;
    st = spai_factor(A_next, A_prev, o, s, P, &Q);
    if (st) {
        delete P;
        return st;
    }
    P->factors = P_prev->factors;
    P->factors.push_back(Q);
    *P_out = P;
    return AIRGA_OK;
}

int airga_precond_apply(airga_precond P, const double *r, double *z, int32_t symmetrize,
                        void *stream) {
    TraceScope trace_("airga_precond_apply", stream);
    if (!P || (P->factors.empty() && P->cfactors.empty()) || !r || !z)
        return fail(AIRGA_E_INVALID_ARG, "bad apply operands");
    cudaStream_t s = S(stream);
    if (P->factors.empty()) return precond_apply_general(P, r, z, symmetrize, s);
    const int64_t n = P->n;
    if (P->factors.size() == 1 && symmetrize && P->psym) {
        AIRGA_CUDA(launch_band_apply(n, P->psym->d, r, z, false, s));
        return AIRGA_OK;
    }
    void *tmp = nullptr;
    int st = dev_alloc(&tmp, sizeof(double) * 3 * (size_t)n, s);
    if (st) return st;
    double *t1 = (double *)tmp, *t2 = t1 + n, *t3 = t2 + n;
    cudaError_t e = cudaSuccess;
    // C r
    const double *src = r;
    for (size_t f = 0; f < P->factors.size() && e == cudaSuccess; ++f) {
        double *dst = (f & 1) ? t2 : t1;
        e = launch_band_apply(n, P->factors[f]->d, src, dst, false, s);
        src = dst;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    if (symmetrize && e == cudaSuccess) {
        // C^T r = F_0^T ... F_last^T r
        src = r;
        size_t cnt = 0;
        for (size_t q = P->factors.size(); q-- > 0 && e == cudaSuccess; ++cnt) {
            double *dst = (cnt & 1) ? t3 : t1;
            e = launch_band_apply(n, P->factors[q]->d, src, dst, true, s);
            src = dst;
        }
        if (e == cudaSuccess) e = launch_axpby(n, 0.5, src, 0.5, z, s);
    }
    dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "precond apply");
    return AIRGA_OK;
}

int32_t airga_precond_length(airga_precond P) {
    return P ? (int32_t)(P->factors.size() + P->cfactors.size()) : 0;
}

int64_t airga_precond_rows(airga_precond P) { return P ? P->n : 0; }

int airga_precond_factor(airga_precond P, int32_t k, double *band, void *stream) {
    if (P && k >= 0 && k < (int32_t)P->cfactors.size() && P->factors.empty())
        return fail(AIRGA_E_UNSUPPORTED,
                    "factor is stored as a general sparse matrix: use airga_precond_factor_csr");
    if (!P || k < 0 || k >= (int32_t)P->factors.size() || !band)
        return fail(AIRGA_E_INVALID_ARG, "bad factor request");
    AIRGA_CUDA(cudaMemcpyAsync(band, P->factors[k]->d, sizeof(double) * kBand * (size_t)P->n,
                               cudaMemcpyDeviceToDevice, S(stream)));
    return AIRGA_OK;
}

int airga_precond_from_bands(int64_t n, int32_t nfactors, const double *const *bands,
                             void *stream, airga_precond *P_out) {
    if (!P_out) return fail(AIRGA_E_INVALID_ARG, "P_out is NULL");
    *P_out = nullptr;
    if (n < 1 || nfactors < 1 || nfactors > kMaxChain || !bands)
        return fail(AIRGA_E_INVALID_ARG, "bad factor list");
    cudaStream_t s = S(stream);
    auto *P = new airga_precond_s;
    P->n = n;
    int st = AIRGA_OK;
    for (int32_t k = 0; k < nfactors && !st; ++k) {
        if (!bands[k]) { st = fail(AIRGA_E_INVALID_ARG, "NULL band"); break; }
        BandPtr b;
        st = make_band(n, s, &b);
        if (st) break;
        cudaError_t e = cudaMemcpyAsync(b->d, bands[k], sizeof(double) * kBand * (size_t)n,
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { st = cuda_fail(e, "copy factor"); break; }
        P->factors.push_back(b);
    }
    if (!st && nfactors == 1) {
        st = make_band(n, s, &P->psym);
        if (!st) {
            cudaError_t e = launch_symmetrize(n, P->factors[0]->d, P->psym->d, s);
            if (e != cudaSuccess) st = cuda_fail(e, "symmetrize");
        }
    }
    if (st) {
        delete P;
        return st;
    }
    *P_out = P;
    return AIRGA_OK;
}

int airga_precond_status(airga_precond P, int32_t *steps, double *colres, int *status_out,
                         void *stream) {
    if (!P) return fail(AIRGA_E_INVALID_ARG, "P is NULL");
    cudaStream_t s = S(stream);
    const size_t n = (size_t)P->n;
    if (steps) {
        if (!P->col_steps) return fail(AIRGA_E_INVALID_ARG, "no per-column data (imported handle)");
        AIRGA_CUDA(cudaMemcpyAsync(steps, P->col_steps.get(), sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    if (colres) {
        if (!P->col_res) return fail(AIRGA_E_INVALID_ARG, "no per-column data (imported handle)");
        AIRGA_CUDA(cudaMemcpyAsync(colres, P->col_res.get(), sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    if (status_out) {
        int32_t f = 0;
        if (P->rank_flag) {
            AIRGA_CUDA(cudaMemcpyAsync(&f, P->rank_flag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            AIRGA_CUDA(cudaStreamSynchronize(s));
        }
        // status word bits: 1 rank-deficient column block (SPAI), 2 non-positive
        // diagonal of A (learned SPAI), 4 tensor-core wait timeout (learned SPAI)
        *status_out = f == 0 ? AIRGA_OK
                             : (f & 4) ? AIRGA_E_TIMEOUT
                             : (f & 2) ? AIRGA_E_INVALID_ARG
                                       : AIRGA_E_RANK;
    }
    return AIRGA_OK;
}

void airga_precond_free(airga_precond P) { delete P; }

}  // extern "C"

// airga_pcg_solve, optionally with the right-hand sides F = scale M V formed
// from a band matrix Mrhs and a block V instead of read from F.
static int pcg_solve_impl(airga_mat A, airga_precond P, const double *F, airga_mat Mrhs,
                          const double *V, double scale, int32_t m, const airga_options *opt,
                          double *X, double *res_hist, int32_t *iters, int32_t *status,
                          double *true_relres, void *stream) {
    int st = check_any(A, "A");
    if (st) return st;
    if (m < 0) return fail(AIRGA_E_INVALID_ARG, "m must be >= 0");
    if (m == 0) return AIRGA_OK;
    if ((!F && !V) || !X || !iters || !status || !true_relres)
        return fail(AIRGA_E_INVALID_ARG, "F (or M and V), X, iters, status and true_relres are required");
    if (Mrhs && Mrhs->n != A->n) return fail(AIRGA_E_SHAPE, "M and A differ in size");
    if (P && (P->n != A->n || (P->factors.empty() && P->cfactors.empty())))
        return fail(AIRGA_E_SHAPE, "P does not match A");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    st = check_options(&o);
    if (st) return st;
    if (!A->band || (P && P->factors.empty()) || (Mrhs && !Mrhs->band)) {
        // general sparse storage somewhere: the CSR kernel (right-hand sides
        // scale M V formed once into a temporary)
        cudaStream_t s = S(stream);
        double *Fmat = nullptr;
        if (Mrhs) {
            st = dev_alloc((void **)&Fmat, sizeof(double) * (size_t)A->n * m, s);
            if (st) return st;
            st = airga_spmv(Mrhs, V, Fmat, m, stream);
            for (int32_t c = 0; c < m && !st && scale != 1.0; ++c) {
                cudaError_t fe = launch_axpby(A->n, 0.0, Fmat + (size_t)c * A->n, scale,
                                              Fmat + (size_t)c * A->n, s);
                if (fe != cudaSuccess) st = cuda_fail(fe, "rhs scale");
            }
            F = Fmat;
        }
        if (!st)
            st = pcg_general(A, P, F, m, o, X, res_hist, iters, status, true_relres,
                             take_fault(AIRGA_FAULT_SKIP_ARRIVAL) ? 1 : 0, s);
        if (Fmat) dev_free(Fmat, s);
        return st;
    }
    const int nf = P ? (int)P->factors.size() : 0;
    if (nf > kMaxChain) return fail(AIRGA_E_INVALID_ARG, "chain too long");
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    const int64_t n = A->n;
    const double *mband = nf == 1 ? (o.symmetrize && P->psym ? P->psym->d : P->factors[0]->d)
                                  : nullptr;
    bool al = aligned16(A->band->d) && (!F || aligned16(F)) && aligned16(X) &&
              (!mband || aligned16(mband));
    for (int f = 0; f < nf; ++f) al = al && aligned16(P->factors[f]->d);   // chain stencils: double2
    PcgPlan plan;
    st = pcg_plan(n, nf, nf == 1 && o.symmetrize, al, dev, &plan, o.sm_share);
    if (st) return st;
    cudaStream_t s = S(stream);
    const bool fused_rhs = Mrhs && plan.kind >= 2;
    double *Fmat = nullptr;           // materialised scale M V when the fallback kernel runs
    if (Mrhs && !fused_rhs) {
        st = dev_alloc((void **)&Fmat, sizeof(double) * (size_t)n * m, s);
        if (st) return st;
        cudaError_t fe = launch_spmv(n, Mrhs->band->d, V, Fmat, m, s);
        if (fe == cudaSuccess && scale != 1.0) {
            for (int32_t c = 0; c < m && fe == cudaSuccess; ++c)
                fe = launch_axpby(n, 0.0, Fmat + (size_t)c * n, scale, Fmat + (size_t)c * n, s);
        }
        if (fe != cudaSuccess) {
            dev_free(Fmat, s);
            return cuda_fail(fe, "rhs M V");
        }
        F = Fmat;
    }

    const int nblk = true_residual_blocks(n);
    const size_t n_pbuf = (size_t)n;
    const size_t n_part = (size_t)2 * 4 * plan.grid;
    const size_t n_res = (size_t)2 * nblk * m;
    const size_t doubles = n_pbuf + plan.scratch_doubles + n_part + n_res;
    const size_t bytes = doubles * sizeof(double) + 256;
    void *ws = nullptr;
    st = dev_alloc(&ws, bytes, s);
    if (st) return st;
    double *base = (double *)ws;
    PcgArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.A = A->band->d;
    a.nf = nf;
    for (int f = 0; f < nf; ++f) a.fac[f] = P->factors[f]->d;
    a.psym = (nf == 1 && o.symmetrize && P->psym) ? P->psym->d : nullptr;
    a.symmetrize = o.symmetrize ? 1 : 0;
    a.tol = o.tol;
    a.maxit = o.maxit;
    a.warm = o.warm_start ? 1 : 0;
    a.timeout_ns = (long long)o.barrier_timeout_ms * 1000000ll;
    a.fault_skip_arrival = take_fault(AIRGA_FAULT_SKIP_ARRIVAL) ? 1 : 0;
    a.place = placement_buffer();
    a.pairz = A->pairz ? (const int32_t *)A->pairz.get() : nullptr;
    if (plan.kind >= 2 && A->pairz) {
        // packed beam entries for the row-pair stencil, made once per matrix
        if (!A->packed) {
            st = make_buf(sizeof(double) * 5 * (size_t)n, s, &A->packed);
            if (st) {
                dev_free(ws, s);
                return st;
            }
            cudaError_t pe = launch_pack_pairs(n, A->band->d, (double *)A->packed.get(), s);
            if (pe != cudaSuccess) {
                dev_free(ws, s);
                return cuda_fail(pe, "pack pairs");
            }
        }
        a.Apk = (const double *)A->packed.get();
    }
    a.pbuf = base;
    a.state = base + n_pbuf;
    a.partials = a.state + plan.scratch_doubles;
    double *res_part = a.partials + n_part;
    unsigned *ctl = (unsigned *)(res_part + n_res);
    a.bar = ctl;
    a.abort_flag = (int *)(ctl + 1);
    cudaError_t e = cudaSuccess;
    // the row-pair kernel computes the true residual in its epilogue
    const bool relres_in_kernel = plan.kind >= 2;
    for (int32_t c = 0; c < m && e == cudaSuccess; ++c) {
        if (fused_rhs) {
            a.b = nullptr;
            a.rhs_M = Mrhs->band->d;
            a.rhs_v = V + (size_t)c * n;
            a.rhs_scale = scale;
        } else {
            a.b = F + (size_t)c * n;
        }
        a.relres = relres_in_kernel ? true_relres + c : nullptr;
        a.x = X + (size_t)c * n;
        a.hist = res_hist ? res_hist + (size_t)c * (o.maxit + 1) : nullptr;
        a.iters = iters + c;
        a.status = status + c;
        e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess) e = launch_pcg(plan, a, s);
    }
    if (e == cudaSuccess && !relres_in_kernel)
        e = launch_true_residual(n, A->band->d, X, F, m, true_relres, res_part, nblk, s);
    dev_free(ws, s);
    if (Fmat) dev_free(Fmat, s);
    if (e != cudaSuccess) return cuda_fail(e, "pcg launch");
    return AIRGA_OK;
}

extern "C" {

int airga_pcg_solve(airga_mat A, airga_precond P, const double *F, int32_t m,
                    const airga_options *opt, double *X, double *res_hist, int32_t *iters,
                    int32_t *status, double *true_relres, void *stream) {
    TraceScope trace_("airga_pcg_solve", stream);
    if (!F) return fail(AIRGA_E_INVALID_ARG, "F is required");
    return pcg_solve_impl(A, P, F, nullptr, nullptr, 1.0, m, opt, X, res_hist, iters, status,
                          true_relres, stream);
}

int airga_pcg_solve_mv(airga_mat A, airga_precond P, airga_mat M, const double *V,
                       double rhs_scale, int32_t m, const airga_options *opt, double *X,
                       double *res_hist, int32_t *iters, int32_t *status, double *true_relres,
                       void *stream) {
    TraceScope trace_("airga_pcg_solve_mv", stream);
    int st = check_any(M, "M");
    if (st) return st;
    if (!V) return fail(AIRGA_E_INVALID_ARG, "V is required");
    if (!std::isfinite(rhs_scale)) return fail(AIRGA_E_INVALID_ARG, "rhs_scale must be finite");
    return pcg_solve_impl(A, P, nullptr, M, V, rhs_scale, m, opt, X, res_hist, iters, status,
                          true_relres, stream);
}

int airga_true_residual(airga_mat A, const double *X, const double *F, int32_t m,
                        double *relres, void *stream) {
    TraceScope trace_("airga_true_residual", stream);
    int st = check_any(A, "A");
    if (st) return st;
    if (m < 0 || (m > 0 && (!X || !F || !relres))) return fail(AIRGA_E_INVALID_ARG, "bad residual operands");
    if (m == 0) return AIRGA_OK;
    cudaStream_t s = S(stream);
    if (!A->band) return true_residual_general(A, X, F, m, relres, s);
    const int nblk = true_residual_blocks(A->n);
    void *tmp = nullptr;
    st = dev_alloc(&tmp, sizeof(double) * 2 * (size_t)nblk * m, s);
    if (st) return st;
    cudaError_t e = launch_true_residual(A->n, A->band->d, X, F, m, relres, (double *)tmp, nblk, s);
    dev_free(tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "true residual");
    return AIRGA_OK;
}

int airga_debug_force_pcg_kernel(int kind) {
    if (kind < 0 || kind > 4) return fail(AIRGA_E_INVALID_ARG, "kernel kind must be 0..4");
    g_forced_kind.store(kind);
    return AIRGA_OK;
}

int airga_debug_record_placement(int32_t *sm_of_cta) {
    g_place.store(sm_of_cta);
    return AIRGA_OK;
}

int airga_debug_set_fault(int fault) {
    if (fault != AIRGA_FAULT_NONE && fault != AIRGA_FAULT_SKIP_ARRIVAL &&
        fault != AIRGA_FAULT_ALLOC && fault != AIRGA_FAULT_LAUNCH)
        return fail(AIRGA_E_INVALID_ARG, "unknown fault");
    g_fault.store(fault);
    return AIRGA_OK;
}

int airga_debug_pool_used(int64_t *bytes) {
    if (!bytes) return fail(AIRGA_E_INVALID_ARG, "bytes is NULL");
    cudaMemPool_t pool = nullptr;
    int st = pool_for_current(&pool);
    if (st) return st;
    uint64_t used = 0;
    AIRGA_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    *bytes = (int64_t)used;
    return AIRGA_OK;
}

int airga_trim(void) {
    cudaMemPool_t pool = nullptr;
    int st = pool_for_current(&pool);
    if (st) return st;
    AIRGA_CUDA(cudaMemPoolTrimTo(pool, 0));
    return AIRGA_OK;
}

}  // extern "C"
