/*
 * airga.h — C ABI of libairga.so: the shifted-system SPAI-preconditioned CG
 * path of "Preconditioned Iterative Solves in Model Reduction of Second Order
 * Linear Dynamical Systems" (Singh, Ahuja, Fassbender; arXiv 1606.01216),
 * written for one NVIDIA GB300 GPU (sm_103a).
 *
 * The path solves a sequence of shifted sparse SPD systems
 *     K_i X = F,   K_i = s_i^2 M + s_i D + K,   D = alpha M + beta K
 * (Eq. 1.1; coefficient matrix of Algorithm 3, Sec. 3.1) by preconditioned CG
 * with a sparse approximate inverse P (Sec. 3.1, Eq. 3.1) built on a fixed
 * sparsity pattern, and the SPAI update P_new = Q P_old of Sec. 3.2 applied as
 * a chain of mat-vecs (Algorithm 5).
 *
 * General conventions
 * -------------------
 * - Every function is plain C; no CUDA or torch type appears.  A `stream`
 *   argument is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued asynchronously on that stream unless a
 *   function says it synchronises; results written to caller buffers are
 *   valid after the stream has been synchronised.
 * - Every raw pointer argument is a DEVICE pointer on the current CUDA
 *   device, owned by the caller, unless stated otherwise.  Vectors and
 *   multi-column blocks are FP64, column-major n x m with leading dimension n.
 * - Handles (airga_mat, airga_precond) are owned by the library and released
 *   with the matching *_free.  Their device storage comes from a
 *   library-owned stream-ordered memory pool on the device that was current
 *   at creation; it is released on the stream that created the handle, so
 *   free a handle before destroying that stream.
 * - A matrix handle has one of two storages, chosen at import:
 *   band-7 diagonals ("DIA") when every entry has |col - row| <= 3:
 *   band[(d+3)*n + i] = A(i, i+d) for d = -3..3, entries outside the matrix
 *   held as 0 (the fast path: node-pair CG kernels, band SPAI plans); or
 *   general sparse CSR (rows sorted, no duplicates) otherwise.  Matrices of
 *   the two storages mix freely in the calls below that say so (a band
 *   operand then takes part with the pattern of its nonzero entries, so a
 *   lumped, diagonal mass matrix stays diagonal; this view is made once per
 *   handle and SYNCHRONISES the stream that makes it); the
 *   mixed-precision, batched, no-alloc and learned-SPAI calls need band
 *   storage and give AIRGA_E_UNSUPPORTED for CSR.
 * - Return value: AIRGA_OK or an AIRGA_E_* code for argument, shape, CUDA or
 *   allocation errors detected when the call is made.  Numerical outcomes of
 *   a solve (converged, iteration cap, breakdown, barrier timeout) are written
 *   per column to device memory (pcg_solve's `status`).  No call aborts the
 *   process or traps the device.  airga_last_error() gives a message for the
 *   last failing call on the calling host thread.
 */
#ifndef AIRGA_H
#define AIRGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes ---------------------------------------------------------- */
#define AIRGA_OK 0
#define AIRGA_E_INVALID_ARG 1   /* bad pointer, size, option or handle */
#define AIRGA_E_SHAPE 2         /* operands of different sizes */
#define AIRGA_E_BREAKDOWN 3     /* CG: (p, A p) <= 0 (A not SPD) or (r, z) zero / not finite */
#define AIRGA_E_MAXIT 4         /* CG: iteration cap reached; X holds the last iterate */
#define AIRGA_E_TIMEOUT 5       /* bounded grid barrier gave up; the solve stopped early */
#define AIRGA_E_RANK 6          /* SPAI: a column least-squares block is rank deficient */
#define AIRGA_E_CUDA 7          /* a CUDA runtime call failed */
#define AIRGA_E_OOM 8           /* device allocation failed */
#define AIRGA_E_UNSUPPORTED 9   /* operation not available for this storage (CSR where band is needed) */

/* SPAI modes */
#define AIRGA_SPAI_QR 0         /* exact fixed-pattern least squares, Householder QR */
#define AIRGA_SPAI_MR 1         /* the paper's minimal-residual iteration (Algorithms 2 / 4) */
#define AIRGA_SPAI_NE 2         /* exact fixed-pattern least squares by the normal equations: the
                                   same minimiser as AIRGA_SPAI_QR (see airga_spai_build) */

typedef struct airga_mat_s *airga_mat;
typedef struct airga_precond_s *airga_precond;
typedef struct airga_batch_s *airga_batch;

/* Options shared by the SPAI and CG calls.  Fill with airga_options_default
 * and change fields; passing NULL where an options pointer is taken means
 * the defaults. */
typedef struct {
    double tol;                 /* CG stops when ||r_k||_2 <= tol ||F(:,c)||_2 (default 1e-10) */
    int32_t maxit;              /* CG iteration cap per column (default 20000) */
    int32_t spai_mode;          /* AIRGA_SPAI_QR (default), AIRGA_SPAI_MR or AIRGA_SPAI_NE */
    double mr_tol;              /* MR: stop a column when ||r|| <= mr_tol (default 0.01, Sec. 5; see mr_relative) */
    int32_t mr_kmax;            /* MR: step cap per column (default 50) */
    int32_t symmetrize;         /* CG applies z = 1/2 (C + C^T) r instead of z = C r (default 1) */
    int32_t pattern_hbw;        /* SPAI pattern: band |i - j| <= pattern_hbw, 0..3 (default 3) */
    int32_t warm_start;         /* CG: nonzero = use X's content on entry as x_0 (default 0: x_0 = 0) */
    int32_t barrier_timeout_ms; /* bound on any single grid-barrier wait (default 2000) */
    int32_t want_colres;        /* SPAI: 1 = keep ||b_j - A m_j|| per column for
                                   airga_precond_status (default); 0 = the normal-equation solver
                                   skips forming it (its residual pass is a quarter of that
                                   solver's FP64 work) and those entries read NaN; the Householder
                                   and MR solvers get it as a by-product and always keep it */
    double inner_tol;           /* mixed precision: FP32 inner solve to ||r_in|| <= inner_tol ||r|| (default 3e-4) */
    int32_t max_outer;          /* mixed precision: FP64 refinement steps per column (default 12) */
    int32_t mr_relative;        /* MR stop test: 0 = ||r|| <= mr_tol, the loop test of Algorithms 2 / 4
                                   (default); 1 = ||r|| <= mr_tol ||b_j||, b_j = e_j (build) or
                                   A_prev e_j (update) — the same for a build, scale-free for an update */
    int32_t sm_share;           /* CG: 1 = a solve may take every SM whole (default).  2 (lead) and
                                   3 (partner): the solve takes half of each SM's registers and shared
                                   memory (the node-pair kernel with r, p in shared memory and x, z/q
                                   in L2, 256 threads, where it applies: even n, aligned operands, no
                                   update chain, n up to about 1.03e6 on GB300), so that a lead and a
                                   partner issued on different streams run side by side, one CTA of
                                   each per SM, and each fills the other's barrier and scalar-chain
                                   gaps on the FP64 pipe.  A lead reserves just over half of an SM's
                                   shared memory, so two of its CTAs never share an SM: an SM holding
                                   two CTAs of one solve would pace that solve's every barrier.  Give
                                   the longer solve 2 and launch it first; run the others as 3 on a
                                   second stream that waits for an event after the lead's
                                   preconditioner and then for airga_stream_hold (about 50 us), so
                                   that every lead CTA is placed before partner work takes SM room */
    int32_t reserved0;          /* 0 */
} airga_options;

void airga_options_default(airga_options *opt);
const char *airga_status_string(int status);
const char *airga_last_error(void);
int airga_version(void);        /* 100 * major + minor */

/* ---------------------------------------------------------------------- */
/* matrices                                                                */
/* ---------------------------------------------------------------------- */

/* Import a square n x n CSR matrix (device arrays: rowptr[n+1] int64 with
 * rowptr[0] = 0 and rowptr[n] = nnz, col[nnz] int32, val[nnz] double; the
 * columns of a row in any order).  Duplicate entries are summed (in input
 * order).  When every entry satisfies |col - row| <= 3 the matrix is stored
 * as band-7 (explicit zeros inside the band kept); otherwise it is kept as
 * general sparse CSR with the rows sorted.  Column indices outside [0, n) or
 * malformed rowptr give AIRGA_E_INVALID_ARG.  SYNCHRONISES `stream` (to read
 * back the validation flag and, for CSR, the sizes).  n >= 1. */
int airga_mat_from_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                       const double *val, void *stream, airga_mat *out);

/* 1 if the matrix is stored as band-7, 0 if as general sparse CSR (or NULL). */
int airga_mat_is_banded(airga_mat A);

/* Stored entries: the CSR nnz, or for a band matrix the entries of its full
 * band pattern inside the matrix (7 n - 12 for n >= 3). */
int64_t airga_mat_nnz(airga_mat A);

/* Copy the matrix as CSR (rows sorted): rowptr[n+1], col[nnz], val[nnz]
 * with nnz = airga_mat_nnz(A); a band matrix is written on its full band
 * pattern.  Any pointer may be NULL to skip that array. */
int airga_mat_to_csr(airga_mat A, int64_t *rowptr, int32_t *col, double *val, void *stream);

/* Import band-7 storage band[7*n] (layout above; entries outside the matrix
 * must be 0).  The data are copied. */
int airga_mat_from_band(int64_t n, const double *band, void *stream, airga_mat *out);

/* Copy a band matrix's band-7 storage into band[7*n] (AIRGA_E_UNSUPPORTED
 * for a CSR matrix). */
int airga_mat_to_band(airga_mat A, double *band, void *stream);

/* Rows of a matrix (0 for NULL). */
int64_t airga_mat_rows(airga_mat A);

void airga_mat_free(airga_mat A);

/* ---------------------------------------------------------------------- */
/* the path                                                                */
/* ---------------------------------------------------------------------- */

/* K(s) = s^2 M + s D + K with D = alpha M + beta K (Eq. 1.1; K_i of
 * Algorithms 3 and 5, Sec. 3).  M and K must have equal n.  *A_out is a new
 * handle: band-7 when both are band matrices; otherwise CSR on the union of
 * the two patterns (one pattern shared by every shift assembled from the
 * same M and K; forming a new union SYNCHRONISES `stream` once, later shifts
 * reuse it).  Each stored entry is fma(s^2 + alpha s, m, (1 + beta s) k).
 * When M and K both come from beam
 * matrices (the Hermite-beam zero structure detected at import) and n is
 * even, the same pass also stores the packed nonzeros the CG kernel reads
 * (5 n doubles owned by the handle), so a later airga_pcg_solve needs no
 * packing pass.  Asynchronous on `stream`. */
int airga_assemble_shifted(airga_mat M, airga_mat K, double alpha, double beta, double s,
                           void *stream, airga_mat *A_out);

/* Y = A X for m columns (X, Y: n x m column-major, distinct buffers); either
 * storage. */
int airga_spmv(airga_mat A, const double *X, double *Y, int32_t m, void *stream);

/* SPAI of Sec. 3.1: P minimising ||I - A P||_F = sum_j ||e_j - A p_j||_2
 * (Eq. 3.1) over matrices whose column j is supported on J_j, the row
 * indices of column j of the sparsity pattern S:
 *   - pattern NULL: S = the pattern of A;
 *   - pattern a matrix handle: S = its stored pattern (values unused); for
 *     a band-7 handle, the pattern of its nonzero entries.
 * For a band A with a band (or NULL) pattern, J_j = {k : |k - j| <= hbw},
 * hbw = opt->pattern_hbw, and P is band-7.  Otherwise P is stored as CSR on
 * S (pattern_hbw is not used) and each column's block is limited to
 * |J_j| <= 32 entries and |I_j| <= 64 rows, I_j the rows of A's columns in
 * J_j (AIRGA_E_INVALID_ARG otherwise); the row sets are computed once per
 * pair of patterns, which SYNCHRONISES `stream` on the first build (later
 * builds on matrices of the same pattern, e.g. every shift of one problem,
 * reuse them).  opt->spai_mode selects the exact per-column least-squares
 * solution (Householder QR of the |I_j| x |J_j| block A(I_j, J_j)) or the
 * paper's MR iteration of Algorithm 2 (initial P = alpha I, alpha =
 * trace(A) / trace(A A^T); direction r restricted to J_j; stop test as
 * opt->mr_relative says; steps capped by opt->mr_kmax).
 * AIRGA_SPAI_NE solves the same least-squares problems as AIRGA_SPAI_QR
 * through G m = A(I_j,J_j)^T b_j, G = (A^T A)(J_j, J_j) taken from one
 * band-13 product for all columns, by L D L^T (about half the FP64 work of
 * the Householder solve).  It applies to band storage with pattern_hbw = 3;
 * elsewhere the QR solver runs.  A column whose Gram block is
 * ill-conditioned (a pivot <= 0, or smallest pivot < 1e-6 x largest
 * diagonal entry) is solved by Householder QR instead, so the result is the
 * QR result to within the rounding of a well-conditioned solve; those
 * columns have steps[j] = 1 in airga_precond_status (0 elsewhere).  It
 * takes 7 n doubles and n int32 of pool scratch for the call.  The new handle
 * holds P and, for CG, P_sym = 1/2 (P + P^T) (on S's pattern, or on its
 * union with the transpose when S is not structurally symmetric).  A rank
 * deficient column block is reported through airga_precond_status. */
int airga_spai_build(airga_mat A, airga_mat pattern, const airga_options *opt, void *stream,
                     airga_precond *P_out);

/* SPAI update of Sec. 3.2 / Algorithm 4: Q minimising
 * ||A_prev - A_next Q||_F = sum_j ||A_prev e_j - A_next q_j||_2 over the same
 * kind of pattern, exact (QR) or by the MR iteration with the initial scaling
 * alpha = 1/2 trace(A_prev^T A_next + A_next^T A_prev) / trace(A_next^T A_next).
 * The new handle is the chain [P_prev's factors..., Q], i.e. the
 * preconditioner Q P_prev of Algorithm 5, applied by mat-vecs and never
 * formed.  The new handle keeps P_prev's factors alive (reference counted),
 * so P_prev may be freed at any time.  When A_prev, A_next and P_prev are all
 * band-7, Q is band-7 on the band pattern of opt->pattern_hbw; otherwise Q
 * is CSR on the pattern of A_next, A_prev must share A_next's pattern
 * (AIRGA_E_SHAPE otherwise; matrices assembled from the same M and K do),
 * and band factors of P_prev are carried over as CSR. */
int airga_spai_update(airga_precond P_prev, airga_mat A_prev, airga_mat A_next,
                      const airga_options *opt, void *stream, airga_precond *P_out);

/* z = 1/2 (C + C^T) r (symmetrize != 0) or z = C r, C = F_last ... F_0 the
 * handle's chain.  r, z: n-vectors, distinct buffers. */
int airga_precond_apply(airga_precond P, const double *r, double *z, int32_t symmetrize,
                        void *stream);

/* Number of factors in the chain (1 for a freshly built SPAI), 0 for NULL. */
int32_t airga_precond_length(airga_precond P);

/* Rows of the preconditioner (0 for NULL). */
int64_t airga_precond_rows(airga_precond P);

/* Copy factor k (0 = the built SPAI P, k >= 1 the update factors Q in
 * order) of a band-7 chain into band[7*n] (AIRGA_E_UNSUPPORTED for a CSR
 * chain: use airga_precond_factor_csr). */
int airga_precond_factor(airga_precond P, int32_t k, double *band, void *stream);

/* 1 if the chain's factors are band-7, 0 if CSR (or NULL). */
int airga_precond_is_banded(airga_precond P);

/* Stored entries of factor k (band factors: their full band pattern). */
int64_t airga_precond_factor_nnz(airga_precond P, int32_t k);

/* Copy factor k as CSR (rows sorted): rowptr[n+1], col[nnz], val[nnz], nnz =
 * airga_precond_factor_nnz(P, k); any pointer may be NULL. */
int airga_precond_factor_csr(airga_precond P, int32_t k, int64_t *rowptr, int32_t *col,
                             double *val, void *stream);

/* Build a CSR chain handle from nfactors CSR matrices (host arrays of
 * nfactors device pointers / sizes, factor 0 first; CSR arrays as for
 * airga_mat_from_csr); the data are copied.  A single factor also gets its
 * symmetric part for CG.  With airga_precond_factor_csr this saves and
 * restores a CSR preconditioner.  SYNCHRONISES `stream`. */
int airga_precond_from_csr(int64_t n, int32_t nfactors, const int64_t *nnz,
                           const int64_t *const *rowptr, const int32_t *const *col,
                           const double *const *val, void *stream, airga_precond *P_out);

/* Build a chain handle from nfactors band-7 arrays (device pointers, each
 * 7*n doubles, factor 0 first); the data are copied.  Together with
 * airga_precond_factor this saves and restores a preconditioner. */
int airga_precond_from_bands(int64_t n, int32_t nfactors, const double *const *bands,
                             void *stream, airga_precond *P_out);

/* Per-column results of the SPAI call that produced the newest factor:
 * steps[n] (int32, MR steps; 0 in QR mode) and colres[n] (double,
 * ||b_j - A m_j||_2 of the column least-squares problem); either may be
 * NULL.  *status_out (host) is AIRGA_OK, AIRGA_E_RANK, or — for a handle
 * made by airga_mlp_spai — AIRGA_E_INVALID_ARG (A has a non-positive or
 * non-finite diagonal entry) or AIRGA_E_TIMEOUT (a bounded tensor-core wait
 * gave up); it SYNCHRONISES `stream` when status_out is not NULL. */
int airga_precond_status(airga_precond P, int32_t *steps, double *colres, int *status_out,
                         void *stream);

void airga_precond_free(airga_precond P);

/* Preconditioned CG (Hestenes-Stiefel) on A X = F for m right-hand sides,
 * each column an independent recurrence (Alg. 3 line 5, Alg. 5 lines 7 and
 * 11; CG chosen for SPD K_i, Sec. 5):
 *   x_0 = 0 (or X on entry if opt->warm_start); r_0 = f - A x_0;
 *   z = M r; p = z; for k = 1..maxit: q = A p; a = (r,z)/(p,q);
 *   x += a p; r -= a q; stop if ||r|| <= tol ||f||; z = M r;
 *   b = (r,z)_new / (r,z)_old; p = z + b p,
 * with M = 1/2 (C + C^T) (opt->symmetrize) or C, C the chain of P.  P may
 * be NULL (M = I).  Outputs (device): X[n*m]; iters[m] (int32, iterations
 * done); status[m] (int32, AIRGA_OK / AIRGA_E_MAXIT / AIRGA_E_BREAKDOWN /
 * AIRGA_E_TIMEOUT); true_relres[m] (||f - A x|| / ||f|| recomputed from X at
 * exit in FP64; NaN for a column whose solve ended in AIRGA_E_TIMEOUT, after
 * which no residual pass runs); res_hist[(maxit+1)*m] (optional, may be NULL: column c holds
 * ||r_k|| / ||f|| for k = 0..iters[c], the rest untouched).  A zero column f
 * gives x = 0, iters = 0, status OK, true_relres 0.  Uses a per-call device
 * workspace from the library pool (about 4 n doubles).  Storage: a band-7 A
 * with a band-7 (or no) preconditioner runs the band kernels; any CSR
 * operand runs the general sparse kernel (vectors in global memory, three
 * grid barriers per iteration and one more per further chain factor, about
 * 9 n doubles of workspace). */
int airga_pcg_solve(airga_mat A, airga_precond P, const double *F, int32_t m,
                    const airga_options *opt, double *X, double *res_hist, int32_t *iters,
                    int32_t *status, double *true_relres, void *stream);

/* ---------------------------------------------------------------------- */
/* batched solves                                                          */
/* ---------------------------------------------------------------------- */

/* Plan nsys independent single-RHS solves A[s] x_s = f_s (each the PCG of
 * airga_pcg_solve, e.g. the shifts x right-hand sides of several beams; the
 * RHS reuse of Algorithms 3/5) for ONE persistent launch.  Each system s gets
 * a group of CTAs, sized so that its rows per CTA stay near rows_per_cta
 * (0 = 4096) and fit shared memory; systems are placed largest cost first on
 * the CTAs that become free first.  cost[s] (host, may be NULL = rows) is
 * the caller's work estimate, e.g. rows x CG iterations of an earlier run —
 * the hook an autotuner uses.  group[s] (host, may be NULL): systems with
 * the same group id (and the same CTA-group size) are scheduled as one job,
 * back to back on one CTA group, e.g. the right-hand sides of one (A, P),
 * which then reuse its bands while they sit in L2; NULL schedules every
 * system on its own.  opt->sm_share 1 (default) plans one CTA slot per SM;
 * 2 or 3 plans two lanes of one slot per SM each (256 threads, at most half
 * an SM's registers and shared memory per CTA; x updated in place and the
 * z/q window in a per-slot device slice, about 6,700 rows per CTA at most).
 * A system's CTA group lies within one lane, so its CTAs sit on distinct SMs,
 * and the two CTAs on an SM belong to different systems, which fill each
 * other's barrier gaps; each job goes to the lane where it can start first.
 * Requirements: every n even, F[s] and X[s]
 * (device, n-vectors) 16-byte aligned, either every P[s] a single factor of
 * matching size or P NULL / every P[s] NULL.  Results of each solve go to the
 * caller's device arrays iters[s], status[s] and relres[s] (true residual).
 * The handles A[s], P[s] and all buffers must outlive the plan.  Uploads the
 * plan and SYNCHRONISES `stream`. */
int airga_batch_create(int32_t nsys, const airga_mat *A, const airga_precond *P,
                       const double *const *F, double *const *X, const double *cost,
                       const int32_t *group, int32_t rows_per_cta, const airga_options *opt,
                       int32_t *iters, int32_t *status, double *relres, void *stream,
                       airga_batch *out);


/* Run the planned solves: one memset and one cooperative launch on `stream`,
 * no allocation (the call may be captured in a CUDA graph and replayed; each
 * replay solves again from x_0 = 0 unless opt->warm_start was set). */
int airga_batch_solve(airga_batch b, void *stream);

/* Plan facts: CTAs, requested and largest rows per CTA, estimated makespan
 * (cost units per CTA).  Any pointer may be NULL. */
int airga_batch_info(airga_batch b, int32_t *grid, int32_t *rows_target, int32_t *rows_max,
                     double *makespan);

void airga_batch_free(airga_batch b);

/* Mixed-precision solve of A X = F (FP32 inner CG inside FP64 iterative
 * refinement): for each column, starting from x = 0,
 *   r = f - A x            in FP64 (true residual; stop when ||r|| <= tol ||f||)
 *   solve A d = r          by preconditioned CG in FP32 — FP32 copies of A
 *                          and of the single-factor preconditioner P_sym (or
 *                          of P itself when opt->symmetrize is 0), FP32
 *                          vectors, FP64 reduction totals — until
 *                          ||r - A d|| <= opt->inner_tol ||r|| or opt->maxit
 *   x = x + d              in FP64,
 * at most opt->max_outer times.  The SPAI (built in FP64) is only rounded to
 * FP32 for the inner applications.  Outputs (device): X[n*m];
 * outer_iters[m] and inner_iters[m] (int32: refinement steps taken and
 * total FP32 CG iterations); status[m] (AIRGA_OK when the FP64 residual
 * reached tol, AIRGA_E_MAXIT when max_outer steps did not, AIRGA_E_BREAKDOWN
 * from an inner solve, AIRGA_E_TIMEOUT when a bounded grid barrier expired);
 * true_relres[m] as for airga_pcg_solve.  P must be NULL (no preconditioner)
 * or a single factor.  Each column is one persistent launch that runs its
 * whole refinement loop (asynchronous on `stream`, no host synchronisation).
 * Uses a per-call workspace from the library pool: FP32 copies of A, of its
 * packed beam entries and of P, plus n floats. */
int airga_pcg_solve_mixed(airga_mat A, airga_precond P, const double *F, int32_t m,
                          const airga_options *opt, double *X, int32_t *outer_iters,
                          int32_t *inner_iters, int32_t *status, double *true_relres,
                          void *stream);

/* AIRGA inner-loop solves (Alg. 1 line 14; Alg. 3 lines 9-12; Alg. 5 lines
 * 15-17): A X = rhs_scale M V for an n x m block V (device, column-major),
 * with the same preconditioner P reused for every new right-hand side.  The
 * product M V is formed inside the solve wherever the right-hand side is
 * read (it is not stored) when the row-pair kernel runs (even n, aligned
 * operands, no update chain); otherwise it is formed once into a temporary
 * first.  Otherwise identical to airga_pcg_solve; true_relres is relative to
 * ||rhs_scale M V(:,c)||.  rhs_scale = -1 gives the moment recurrence
 * X = -(s^2 M + s D + K)^{-1} M V of Algorithm 1. */
int airga_pcg_solve_mv(airga_mat A, airga_precond P, airga_mat M, const double *V,
                       double rhs_scale, int32_t m, const airga_options *opt, double *X,
                       double *res_hist, int32_t *iters, int32_t *status, double *true_relres,
                       void *stream);

/* relres[c] = ||F(:,c) - A X(:,c)||_2 / ||F(:,c)||_2 (0 when F(:,c) = 0),
 * the FP64 acceptance residual of a solve. */
int airga_true_residual(airga_mat A, const double *X, const double *F, int32_t m,
                        double *relres, void *stream);

/* Allocation-free variant of airga_pcg_solve.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory — an application whose device memory is entirely owned by
 * its own allocator (a framework that reserves the GPU up front and forbids
 * allocations behind its back), or a latency-critical loop that cannot take
 * the synchronisation and failure point of an allocation call.  It calls no
 * cudaMalloc/cudaFree or other allocating routine.
 *
 * Inputs are raw band-7 arrays instead of handles: A_band[7*n] (the shifted
 * matrix) and M_band[7*n] (the preconditioner, applied exactly as given:
 * z = M r with all seven diagonals read, so M need not be symmetric — pass
 * P_sym = 1/2 (P + P^T) of a SPAI to get airga_pcg_solve's default
 * operator; NULL = no preconditioner), all device memory owned by the
 * caller; F, X, res_hist, iters, status, true_relres and the options mean the
 * same as for airga_pcg_solve (chains of update factors are not accepted
 * here; opt->symmetrize is ignored).
 *
 * Its scratch is a fixed array of 16.2 MiB in the library's device image,
 * which every GPU that loads the library holds until the process exits.
 * Limits: n <= 1048576 rows, and the solve must fit one of the plans that
 * keep their windows in shared memory or in that array (true on a GB300 for
 * every n up to the limit); larger problems give AIRGA_E_INVALID_ARG with an
 * explanatory airga_last_error().  The first call on each device
 * looks up the array's device address (once per device, with that device
 * current); make that first call before any stream capture.  All calls share
 * the array and it keeps the previous call's contents (the barrier words are
 * cleared on the stream before each column), so calls whose GPU work
 * overlaps — on concurrent streams or from several host threads — race and
 * must be serialised by the caller. */
int airga_pcg_solve_noalloc(int64_t n, const double *A_band, const double *M_band,
                            const double *F, int32_t m, const airga_options *opt, double *X,
                            double *res_hist, int32_t *iters, int32_t *status,
                            double *true_relres, void *stream);

/* ---------------------------------------------------------------------- */
/* learned SPAI-column predictor                                           */
/* ---------------------------------------------------------------------- */

/* A small perceptron that predicts the seven entries of SPAI column j
 * (Sec. 3.1, Eq. 3.1, pattern J_j = {j-3..j+3}) of a shifted matrix
 * A = s^2 M + s D + K (Eq. 1.1) from local features, trained on columns of
 * SPAIs built by airga_spai_build.  It stands in for the SPAI update of
 * Sec. 3.2 (a new preconditioner for a new shift at far lower cost than a
 * build); a caller that needs a guarantee solves with it under an iteration
 * cap and falls back to airga_spai_build.
 *
 * Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, relu(z) = max(z, 0),
 * 16 -> 64 -> 64 -> 16
 * (outputs 7..15 unused).  FP32 master parameters, BF16 copies of the
 * weights and BF16 activations as tensor-core operands, FP32 accumulation,
 * FP32 biases and activation functions.  Parameter vector (FP32,
 * AIRGA_MLP_NPARAM values): W1[64][16] | b1[64] | W2[64][64] | b2[64] |
 * W3[16][64] | b3[16], W[out][in] row-major.
 *
 * Features of column j of an n-row A (FP32 rows of 16):
 *   log10(s)/4, alpha, beta, log10(A_jj)/8,
 *   A(j+d, j) / sqrt(A(j+d, j+d) A_jj) for d = -3,-2,-1,1,2,3 (0 outside),
 *   min(j, 8)/8, min(n-1-j, 8)/8, j mod 2, 0, 0, 0.
 * Targets (FP32 rows of 8): t_o = P(j+d, j) sqrt(A(j+d, j+d) A_jj) for
 * d = o - 3, o = 0..6, t_7 = 0; mask byte: bit o set when 0 <= j+d < n.
 * Loss: L = 1/(2B) sum over the B samples of a minibatch and the masked
 * outputs of (y_o - t_o)^2.  Training: Adam (Kingma and Ba 2015) with bias
 * correction, optional half-cosine learning-rate decay. */
#define AIRGA_MLP_IN 16
#define AIRGA_MLP_HIDDEN 64
#define AIRGA_MLP_OUT 16
#define AIRGA_MLP_NPARAM 6288

typedef struct airga_mlp_s *airga_mlp;

typedef struct {
    float lr;                   /* Adam step size (default 2e-3) */
    float beta1, beta2, eps;    /* Adam moments (defaults 0.9, 0.999, 1e-8) */
    int32_t batch;              /* samples per step (default 4096) */
    int32_t cosine_steps;       /* > 0: lr_t = lr (1 + cos(pi min(t, c) / c)) / 2 at Adam step t (default 0 = constant) */
    uint64_t seed;              /* minibatch draw: sample k of step t is SplitMix64 output number
                                   t * 2^32 + k of the sequence started at seed, modulo count */
} airga_mlp_train_options;

void airga_mlp_train_options_default(airga_mlp_train_options *opt);

/* New network with Glorot-uniform weights drawn from SplitMix64(seed) on the
 * host and zero biases; Adam state zero.  SYNCHRONISES `stream`.  The handle
 * owns about 0.1 MB plus a gradient scratch of 25 KB per SM. */
int airga_mlp_create(uint64_t seed, void *stream, airga_mlp *out);

/* Copy AIRGA_MLP_NPARAM FP32 parameters in from device memory and reset the
 * Adam state and the step counter. */
int airga_mlp_set_params(airga_mlp net, const float *params, void *stream);

/* Copy the AIRGA_MLP_NPARAM FP32 master parameters out to device memory. */
int airga_mlp_get_params(airga_mlp net, float *params, void *stream);

/* Adam steps taken so far and an error status (AIRGA_OK, AIRGA_E_INVALID_ARG
 * for an out-of-range sample index, AIRGA_E_TIMEOUT for a tensor-core wait
 * that gave up).  SYNCHRONISES `stream`. */
int airga_mlp_status(airga_mlp net, int64_t *steps_done, int *status_out, void *stream);

/* Training pairs from a shifted matrix A (shift s > 0, damping alpha, beta)
 * and, optionally, its SPAI P (a single-factor handle, e.g. from
 * airga_spai_build): for the columns cols[0..count) (device int64; NULL =
 * columns 0..count-1, count <= n) write X[count][16] and, when P is given,
 * T[count][8] and mask[count].  X and T are 16-byte aligned device arrays.
 * *flag (device int32, caller-zeroed) gets bit 8 for a column index outside
 * [0, n) (that row is skipped) and bit 2 for a non-positive diagonal. */
int airga_mlp_features(airga_mat A, airga_precond P, double s, double alpha, double beta,
                       const int64_t *cols, int64_t count, float *X, float *T, uint8_t *mask,
                       int32_t *flag, void *stream);

/* Y[count][16] = network outputs for the feature rows X[count][16]
 * (tensor-core inference kernel; X, Y 16-byte aligned). */
int airga_mlp_forward(airga_mlp net, const float *X, int64_t count, float *Y, void *stream);

/* Mean gradient dL/dparams (grad: AIRGA_MLP_NPARAM floats, device) and loss
 * (*loss, device double, may be NULL) over the minibatch idx[0..batch)
 * (device int32 row indices into X, T, mask; count <= 2^31 - 1) at the
 * current parameters; nothing is updated. */
int airga_mlp_grad(airga_mlp net, const float *X, const float *T, const uint8_t *mask,
                   int64_t count, const int32_t *idx, int32_t batch, float *grad, double *loss,
                   void *stream);

/* `steps` Adam steps on the training set (X, T, mask; count rows), each one
 * forward/backward launch and one update launch, enqueued without host
 * synchronisation (graph-capturable; the step counter lives on the device).
 * idx: NULL = draw minibatches on the device (opt->seed), else device int32
 * [steps * batch] explicit indices.  loss_hist (device, may be NULL) gets
 * the loss of each step's minibatch before its update. */
int airga_mlp_train(airga_mlp net, const float *X, const float *T, const uint8_t *mask,
                    int64_t count, int32_t steps, const airga_mlp_train_options *opt,
                    const int32_t *idx, float *loss_hist, void *stream);

/* Learned SPAI for A = s^2 M + s D + K: the network's outputs for every
 * column, unscaled, as a band-7 factor P (entries outside the matrix 0),
 * plus P_sym = 1/2 (P + P^T), in a new single-factor handle usable wherever
 * a built SPAI is (airga_pcg_solve, airga_batch_create, ...).  Per-column
 * SPAI data (steps, colres) are not produced.  Errors found on the device
 * are reported by airga_precond_status. */
int airga_mlp_spai(airga_mlp net, airga_mat A, double s, double alpha, double beta, void *stream,
                   airga_precond *P_out);

void airga_mlp_free(airga_mlp net);

/* Test hook for failure detection (no GPU fault involved): arm a fault for
 * the next airga_pcg_solve, airga_pcg_solve_mixed or airga_batch_solve call
 * of this process.  AIRGA_FAULT_SKIP_ARRIVAL makes CTA 0 (of system 0, in a
 * batch) skip its arrival at the first (inner) iteration barrier of the
 * first column, so every bounded barrier wait of that system
 * (opt->barrier_timeout_ms) expires and its status is AIRGA_E_TIMEOUT; the
 * other systems of a batch, the kernel and the CUDA context carry on.  The
 * fault is consumed by that call.  Two more faults are host-side only and
 * are consumed by the next call that reaches their point:
 * AIRGA_FAULT_ALLOC makes the next device allocation of the library fail
 * (the call returns AIRGA_E_OOM); AIRGA_FAULT_LAUNCH makes the next PCG or
 * SPAI kernel launch report a launch failure (AIRGA_E_CUDA, nothing is
 * launched).  Either way the call releases what it had allocated and later
 * calls work normally. */
#define AIRGA_FAULT_NONE 0
#define AIRGA_FAULT_SKIP_ARRIVAL 1
#define AIRGA_FAULT_ALLOC 2
#define AIRGA_FAULT_LAUNCH 3
int airga_debug_set_fault(int fault);

/* Test hook: bytes of the library's device pool in use on the current
 * device (allocations not yet released; after a stream synchronise this
 * shows leaks). */
int airga_debug_pool_used(int64_t *bytes);

/* Bounds-checked builds.  The library compiled with -DAIRGA_CHECKED
 * (libairga_checked.so beside libairga.so) tests every instrumented index of
 * its PCG, mixed-precision, SPAI and general-sparse kernels against the
 * buffer it addresses before the access: window and band rows, row
 * pointers, column indices, transposition maps and factor positions.  An
 * index outside is counted and the access skipped (a load reads 0), so a
 * wrong index shows up as a count instead of a memory fault.
 *
 * airga_debug_checked waits for the device, then writes the number of
 * violations since the last call to *violations (host) and, when non-zero,
 * the check site and offending index of one of them to *first_site and
 * *first_index (host, may be NULL); the record is then cleared.  Normal
 * builds set *violations to 0 and return AIRGA_E_UNSUPPORTED.
 *
 * airga_debug_check_selftest launches one thread on `stream` that tests
 * `index` against [0, bound) with the kernels' check and touches no memory
 * at `index` (any value is safe); an index outside is recorded with `site`.
 * Normal builds return AIRGA_E_UNSUPPORTED. */
int airga_debug_checked(int64_t *violations, int32_t *first_site, int64_t *first_index);
int airga_debug_check_selftest(int64_t index, int64_t bound, int32_t site, void *stream);

/* Test hook: make the CG calls of this process (airga_pcg_solve,
 * airga_pcg_solve_mv) use one kernel variant whenever it is applicable, so
 * that every variant can be checked on small problems.  0 = automatic (the
 * default): the node-pair kernel with the whole solve state in shared memory
 * when even n fits, else the node-pair kernel with the r and p windows in
 * shared memory and x, z/q in global memory, else the generic kernel.
 * 1 = generic kernel with its state in global memory, 2 = node-pair kernel
 * with shared-memory state, 3 = node-pair kernel with split state, 4 = the
 * split-state kernel on half an SM (256 threads, two CTAs per SM: two solves
 * on different streams share the SMs).  A variant that does not apply (odd
 * n, unaligned operands, update chains, too little shared memory) falls
 * through to the next one as in automatic mode. */
#define AIRGA_PCG_KERNEL_AUTO 0
#define AIRGA_PCG_KERNEL_GENERIC_GLOBAL 1
#define AIRGA_PCG_KERNEL_PAIR 2
#define AIRGA_PCG_KERNEL_PAIR_SPLIT 3
#define AIRGA_PCG_KERNEL_PAIR_HALF 4
int airga_debug_force_pcg_kernel(int kind);

/* Test hook: while `sm_of_cta` (device, at least as many int32 as the GPU
 * has SMs) is set, every CG call that runs a node-pair kernel writes the SM
 * index of each of its CTAs there, CTA rank k at sm_of_cta[k]; NULL (the
 * default) turns it off.  The pointer is read when a call is made, so each
 * of two concurrent solves can be given its own buffer.  airga_batch_create
 * reads it too: every solve of a plan created while it is set writes system
 * s's CTA rank k at sm_of_cta[s * 1024 + k] (the buffer then needs 1024 int32
 * per system). */
int airga_debug_record_placement(int32_t *sm_of_cta);

/* Scheduling aid for lead / partner solves (options.sm_share 2 and 3), no
 * counterpart in the paper: queue on `stream` one warp that sleeps for
 * `microseconds` (0..1000) by the GPU's global timer.  Placed on the
 * partners' stream after the event that releases it, it keeps partner work
 * off the SMs while the lead's CTAs are placed (a cooperative grid is placed
 * CTA by CTA, so partner CTAs arriving meanwhile can take the room of a lead
 * CTA, which then waits for them at the lead's first barrier). */
int airga_stream_hold(int32_t microseconds, void *stream);

/* Measurement aid, no counterpart in the paper: the FP64 FMA issue rate of
 * the current device, the roofline of this library's FP64-bound kernels.
 * One CTA of 1024 threads per SM runs 8, 12 and then 16 independent FMA
 * chains per thread for `iters` steps (1..2^24); *fma_per_clk_sm (host)
 * receives the best of the three in FMAs per SM clock from the SMs' cycle
 * counters (median over SMs, clock independent),
 * *tflops and *ms (host, may be NULL) the rate and time by events at the
 * clocks of the moment.  SYNCHRONISES `stream`. */
int airga_probe_fp64_rate(int64_t iters, double *fma_per_clk_sm, double *tflops, double *ms,
                          void *stream);

/* Measurement aid, no counterpart in the paper: read bandwidth of a device
 * buffer of `bytes` (a multiple of 16 in [1 MiB, 16 GiB]; below the L2 size
 * this is the L2 read bandwidth, above it DRAM's).  4 CTAs of 512 threads
 * per SM stream 16-byte loads that bypass L1 over the buffer (from the
 * library pool, filled first); one untimed pass warms the cache, then
 * `passes` (1..1000) passes run in one timed launch.  *gbs (host) receives
 * bytes x passes / time in GB/s, *ms (host, may be NULL) the time.
 * SYNCHRONISES `stream`. */
int airga_probe_read_bw(int64_t bytes, int32_t passes, double *gbs, double *ms, void *stream);

/* Release the library's cached device memory (pool trim) on the current
 * device; outstanding handles stay valid. */
int airga_trim(void);

/* Call tracing, no counterpart in the paper.  While enabled, each traced
 * call (matrix import, assemble_shifted, spmv, spai_build, spai_update,
 * precond_apply, the pcg_solve family except the allocation-free one,
 * true_residual, batch_solve, mlp_train, mlp_forward, mlp_spai) records a
 * CUDA event on its stream before it enqueues work and another when it
 * returns; the elapsed device time between them covers the work that call
 * enqueued (and any work queued before it on the same stream that was still
 * running).  Calls on a stream under graph capture are not traced.
 *
 * airga_trace_enable(capacity): capacity 1..2^24 turns tracing on and keeps
 * at most that many unread records (later calls are counted as dropped);
 * 0 turns it off and discards unread records.  Host-side state, shared by
 * every thread of the process. */
typedef struct {
    const char *name;   /* the entry point's name (static storage) */
    double ms;          /* device time between the call's two events */
    void *stream;       /* the call's stream */
} airga_trace_record;
int airga_trace_enable(int32_t capacity);

/* Move up to `max_records` of the oldest unread records into `out` (host
 * array), oldest first; *count (host) receives how many.  Waits for each
 * record's end event.  *dropped (host, may be NULL) receives the number of
 * calls not recorded for lack of capacity since the previous read, and that
 * count restarts at 0. */
int airga_trace_read(airga_trace_record *out, int32_t max_records, int32_t *count,
                     int64_t *dropped);

#ifdef __cplusplus
}
#endif

#endif /* AIRGA_H */
