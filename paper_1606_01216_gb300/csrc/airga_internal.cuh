// Internal declarations of libairga (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/airga.h"

namespace airga {

constexpr int kBand = 7;   // diagonals -3..+3
constexpr int kHalf = 3;

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define AIRGA_CUDA(call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// device memory: one stream-ordered pool per device, owned by the library
// ---------------------------------------------------------------------------
int dev_alloc(void **p, size_t bytes, cudaStream_t s);
int check_options(const airga_options *o);
// shared_ptr<void> owning a pool allocation (freed on `s`, on its device)
int make_buf(size_t bytes, cudaStream_t s, std::shared_ptr<void> *out);
int check_mat(airga_mat A, const char *name);
bool aligned16(const void *p);
void dev_free(void *p, cudaStream_t s);

// A band-7 array of 7*n doubles, freed on its creation stream.
struct Band {
    int64_t n = 0;
    double *d = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    ~Band();
};
using BandPtr = std::shared_ptr<Band>;
int make_band(int64_t n, cudaStream_t s, BandPtr *out);

// A sparsity pattern in CSR form together with its transpose (CSC) and the
// map between the two, on the device; shared by every matrix and factor with
// that structure (assemble_shifted keeps it, so the per-shift matrices of
// one problem share one pattern).  Column indices are sorted within rows,
// row indices within columns, no duplicates.
struct CsrPat {
    int64_t n = 0, nnz = 0;
    int64_t *rowptr = nullptr;   // [n+1], rowptr[0] = 0
    int32_t *col = nullptr;      // [nnz]
    int64_t *colptr = nullptr;   // [n+1]
    int32_t *rowidx = nullptr;   // [nnz]
    int64_t *tperm = nullptr;    // [nnz]: CSR index of CSC entry f
    int32_t max_row = 0, max_col = 0;   // longest row / column (host copies)
    bool symmetric = false;      // structurally symmetric: CSC arrays equal the CSR arrays
    std::shared_ptr<void> mem;   // owns the arrays
    // symbolic SPAI data, made on the first SPAI with this pattern as the
    // matrix: keyed by the pattern S whose columns are J_j
    struct Rows {
        std::weak_ptr<CsrPat> S;             // the pattern the sets belong to
        std::shared_ptr<void> buf;           // owns iptr and irows
        const int64_t *iptr = nullptr;       // [n+1]
        const int32_t *irows = nullptr;      // [iptr[n]]: I_j, sorted
        int32_t max_i = 0, max_j = 0;
    };
    std::vector<Rows> spai_rows;
    // cached union patterns with other patterns (assemble_shifted of matrices
    // with different structure; the symmetric part of a factor on a
    // structurally nonsymmetric pattern)
    struct Union {
        std::weak_ptr<CsrPat> other;
        bool other_transposed = false;
        std::shared_ptr<CsrPat> result;
    };
    std::vector<Union> unions;
};
using CsrPatPtr = std::shared_ptr<CsrPat>;

}  // namespace airga

struct airga_mat_s {
    int64_t n = 0;
    airga::BandPtr band;
    // general sparse storage (band == nullptr): pattern + values in CSR order
    airga::CsrPatPtr csr;
    std::shared_ptr<void> cval;          // double[csr->nnz]
    // device int32: nonzero when every row pair (2k, 2k+1) but the last has the
    // Hermite-beam zeros (even rows: offsets -3, +1; odd rows: +3, -1)
    std::shared_ptr<void> pairz;
    // packed copy of the beam's nonzero entries for the PCG row-pair stencil
    // (5 doubles per row, made on the first solve with this matrix)
    std::shared_ptr<void> packed;
};

namespace airga {
// One CSR factor of a preconditioner chain: pattern (with its transpose, for
// C^T r) and values in CSR order.
struct CsrFactor {
    CsrPatPtr pat;
    std::shared_ptr<void> val;
    const double *v() const { return (const double *)val.get(); }
};
}  // namespace airga

struct airga_precond_s {
    int64_t n = 0;
    std::vector<airga::BandPtr> factors;  // factor 0 = built P, then Q_2, Q_3, ...
    airga::BandPtr psym;                  // 1/2 (P + P^T) when factors.size() == 1
    // general sparse chain (factors empty): CSR factors and, for a single
    // factor, its symmetric part
    std::vector<airga::CsrFactor> cfactors;
    airga::CsrFactor csym;
    // per-column results of the SPAI call that made the newest factor
    std::shared_ptr<void> col_steps;      // int32[n]
    std::shared_ptr<void> col_res;        // double[n]
    std::shared_ptr<void> rank_flag;      // int32[1]
};

namespace airga {

// ---------------------------------------------------------------------------
// kernel launchers (band_kernels.cu)
// ---------------------------------------------------------------------------
cudaError_t launch_csr_to_band(int64_t n, const int64_t *rowptr, const int32_t *col,
                               const double *val, double *band, int32_t *flag, cudaStream_t s);
// n even; packed: 5 n doubles, written when both flags are set
cudaError_t launch_assemble_pack(int64_t n, const double *M, const double *K, double alpha,
                                 double beta, double sh, double *A, double *packed, cudaStream_t s,
                                 const int32_t *fm, const int32_t *fk, int32_t *fa);
cudaError_t launch_assemble(int64_t n, const double *M, const double *K, double alpha,
                            double beta, double sh, double *A, cudaStream_t s,
                            const int32_t *fm = nullptr, const int32_t *fk = nullptr,
                            int32_t *fa = nullptr);
// packed[k n + i], packed[k n + i + 1] (i even, k = 0..4): entries of rows
// i and i+1 at offsets (-2,-1,0,+2,+3) and (-3,-2,0,+1,+2) — the nonzeros of
// the beam row pair (n even)
cudaError_t launch_pack_pairs(int64_t n, const double *band, double *packed, cudaStream_t s);
// beam zero-structure flag of a band (flag must be preset to nonzero)
cudaError_t launch_detect_pairz(int64_t n, const double *band, int32_t *flag, cudaStream_t s);
cudaError_t launch_spmv(int64_t n, const double *band, const double *X, double *Y, int32_t m,
                        cudaStream_t s);
cudaError_t launch_band_apply(int64_t n, const double *band, const double *x, double *y,
                              bool transpose, cudaStream_t s);
cudaError_t launch_symmetrize(int64_t n, const double *P, double *Psym, cudaStream_t s);
cudaError_t launch_axpby(int64_t n, double a, const double *x, double b, double *y,
                         cudaStream_t s);
// relres[c] = ||F_c - A X_c|| / ||F_c||; `partial` holds 2 * nblk * m doubles
cudaError_t launch_true_residual(int64_t n, const double *band, const double *X,
                                 const double *F, int32_t m, double *relres, double *partial,
                                 int nblk, cudaStream_t s);
int true_residual_blocks(int64_t n);
// Frobenius-type sums for the MR initial scaling: out[0] = sum a_ii (or
// <A_old, A_new>_F), out[1] = ||A||_F^2 (or ||A_new||_F^2), then out[2] = alpha0
cudaError_t launch_mr_alpha(int64_t n, const double *A, const double *A_old, double *partial,
                            int nblk, double *out, cudaStream_t s);
int mr_alpha_blocks(int64_t n);

// ---------------------------------------------------------------------------
// SPAI (spai_kernels.cu)
// ---------------------------------------------------------------------------
// QR mode: exact LS per column.  A_old == nullptr -> SPAI (b_j = e_j), else
// update (b_j = A_old e_j).  Output band-7 factor F (entries outside the
// pattern 0).  colres: ||b_j - A m_j|| per column.  rank_flag set on a
// rank-deficient column block.
// zA, zAold: device beam zero-structure flags of A and A_old (may be null);
// when set, interior columns skip the structural zeros of their blocks.
cudaError_t launch_spai_qr(int64_t n, int hbw, const double *A, const double *A_old, double *F,
                           double *colres, int32_t *rank_flag, const int32_t *zA,
                           const int32_t *zAold, cudaStream_t s);
// MR mode (Algorithms 2 / 4); alpha0 read from device memory.  A column
// stops when ||r|| <= tol (relative == 0) or ||r|| <= tol ||b_j||.
cudaError_t launch_spai_mr(int64_t n, int hbw, const double *A, const double *A_old,
                           const double *alpha0, double tol, int relative, int kmax, double *F,
                           int32_t *steps, double *colres, cudaStream_t s);
// Normal-equations mode (half-width 3): Gram band of A^T A into U (7 n
// doubles of scratch), L D L^T per column; columns whose Gram block is
// ill-conditioned are solved by the Householder kernel instead and marked
// steps[j] = 1 (steps zeroed by the caller).  fb: n + 1 int32 of scratch.
// want_colres false: the NE columns' colres entries are set to NaN instead
// of forming the residual (the Householder columns still write theirs).
// zA (device, may be null): A's beam-structure flag; when set the column
// kernel skips the Gram block's zero corner.
cudaError_t launch_spai_ne(int64_t n, const double *A, const double *A_old, double *F,
                           double *colres, bool want_colres, int32_t *rank_flag, int32_t *steps,
                           double *U, int32_t *fb, const int32_t *zA, cudaStream_t s);

// ---------------------------------------------------------------------------
// general sparse storage (csr_kernels.cu, spai_csr.cu, pcg_csr.cu)
// ---------------------------------------------------------------------------
struct RowView;
// canonical copy of a caller's CSR (rows sorted, duplicates summed in input
// order) with its pattern; SYNCHRONISES s.  Arrays must be validated first.
int csr_import(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
               const double *val, cudaStream_t s, CsrPatPtr *pat, std::shared_ptr<void> *vals);
// pattern of the full band |i - j| <= 3 (7 n - 12 entries for n >= 4); SYNCHRONISES s
int band_pattern(int64_t n, cudaStream_t s, CsrPatPtr *out);
// values of a band-7 array on band_pattern(n)
cudaError_t launch_band_values(const CsrPat &p, const double *band, double *val, cudaStream_t s);
// the nonzero entries of a band-7 array as CSR with its own pattern; SYNCHRONISES s
int band_nonzero_csr(int64_t n, const double *band, cudaStream_t s, CsrPatPtr *pat,
                     std::shared_ptr<void> *vals);
// equal n, nnz, rowptr and col; SYNCHRONISES s (unless sizes differ)
int csr_same_structure(const CsrPat &a, const CsrPat &b, cudaStream_t s, bool *same);
// union of the row patterns of X and Y; SYNCHRONISES s
int csr_union(int64_t n, const RowView &X, const RowView &Y, cudaStream_t s, CsrPatPtr *out);
// Z = a X + b Y on Z's pattern (a superset of both), fma(a, x, b y) per entry
cudaError_t launch_csr_add(const CsrPat &Z, double a, const RowView &X, double b,
                           const RowView &Y, double *val, cudaStream_t s);
cudaError_t launch_csr_spmv(int64_t n, const RowView &A, const double *X, double *Y, int32_t m,
                            cudaStream_t s);
int csr_blocks(int64_t n);
// relres[c] = ||F_c - A X_c|| / ||F_c||; `partial` holds 2 * nblk * m doubles
cudaError_t launch_csr_true_residual(int64_t n, const RowView &A, const double *X,
                                     const double *F, int32_t m, double *relres,
                                     double *partial, int nblk, cudaStream_t s);
// out[0..2] as launch_mr_alpha, over the stored entries (A_old on A's pattern)
cudaError_t launch_csr_mr_alpha(const CsrPat &p, const double *A, const double *A_old,
                                double *partial, int nblk, double *out, cudaStream_t s);

// Symbolic SPAI: the row sets I_j (rows of A's columns in J_j, J_j = column
// j of S) of every column, cached on A's pattern (SYNCHRONISES s the first
// time for a pattern pair).  AIRGA_E_INVALID_ARG when a column exceeds the
// kernel's limits (|J_j| <= kSpaiMaxJ, |I_j| <= kSpaiMaxI).
constexpr int kSpaiMaxJ = 32, kSpaiMaxI = 64;
int csr_spai_rows(const CsrPatPtr &A, const CsrPatPtr &S, cudaStream_t s,
                  const CsrPat::Rows **out);
// Numeric SPAI on a general pattern, one warp per column: QR (mr == 0) or
// the MR iteration (mr != 0; alpha0 on the device).  A_old (values on A's
// pattern) selects the update right-hand side A_old e_j.  F: values on S's
// pattern in CSR order.  flag bit 1: rank-deficient column block.
cudaError_t launch_spai_csr(const CsrPat &A, const double *Av, const double *Aold,
                            const CsrPat &S, const CsrPat::Rows &rows, int mr,
                            const double *alpha0, double tol, int relative, int kmax, double *F,
                            int32_t *steps, double *colres, int32_t *flag, cudaStream_t s);

// ---------------------------------------------------------------------------
// persistent PCG (pcg_kernel.cu)
// ---------------------------------------------------------------------------
constexpr int kMaxChain = 16;

struct PcgPlan {
    int kind = 0;          // 0 generic (shared-memory state), 1 generic (global state), 2 node-pair,
                           // 3 node-pair with r, p in shared memory and x, z/q in global memory,
                           // 4 the same on half an SM (two solves side by side)
    int grid = 0;          // CTAs (all co-resident)
    int threads = 0;
    int64_t rows = 0;      // rows per CTA (R)
    int halo = 0;          // r window halo H
    bool smem_state = false;
    size_t smem_bytes = 0;
    size_t scratch_doubles = 0;  // global workspace (doubles), excluding the control block
};

struct PcgArgs {
    int64_t n;
    const double *A;
    int nf;                        // chain length (0 = identity preconditioner)
    const double *fac[kMaxChain];  // factor bands, factor 0 first
    const double *psym;            // precomputed symmetric factor (nf == 1 && symmetrize) or null
    int symmetrize;
    const double *b;
    double *x;
    double tol;
    int maxit;
    int warm;
    double *hist;                  // (maxit+1) or null
    int32_t *iters;
    int32_t *status;
    long long timeout_ns;
    // workspace
    double *pbuf;                  // n doubles (boundary rows of p)
    double *rbuf;                  // 2 n doubles (boundary rows of r, double buffered)
    double *state;                 // per-CTA window state when it is not in shared memory
    double *partials;              // 2 slots x 4 values x grid
    unsigned int *bar;             // barrier counter (zeroed before launch)
    int *abort_flag;               // set by a CTA whose barrier wait timed out
    int fault_skip_arrival;        // test injection: CTA 0 skips its first iteration barrier
    const int32_t *pairz;          // device flag: A has the beam zero structure (may be null)
    const double *Apk;             // packed beam entries of A (launch_pack_pairs) or null
    double *relres;                // node-pair kernel: true residual written here (or null)
    const double *rhs_M;           // node-pair kernel: b = rhs_scale M v formed on the fly (or null)
    const double *rhs_v;
    double rhs_scale;
    int32_t *place = nullptr;      // test hook: node-pair kernels write each CTA's SM id here
};

// process-wide test fault consumed by the next pcg_solve (airga_debug_set_fault)
// (consumes it and returns true when the armed fault is `kind`)
bool take_fault(int kind);
// cudaErrorLaunchOutOfResources when AIRGA_FAULT_LAUNCH is armed (consumed),
// else cudaSuccess: called where a solve or SPAI kernel is about to launch
cudaError_t injected_launch_error();
// test hook (airga_debug_record_placement): device buffer for the next CG
// call's CTA placement, or null
int32_t *placement_buffer();

// Call tracing (airga_trace_enable): declare one at the top of a traced
// C-ABI call; it records an event on `stream` now and another when the call
// returns, when tracing is on and the stream is not being captured.
class TraceScope {
  public:
    TraceScope(const char *name, void *stream);
    ~TraceScope();
    TraceScope(const TraceScope &) = delete;
    TraceScope &operator=(const TraceScope &) = delete;

  private:
    const char *name_;
    void *stream_;
    void *e0_;
};

// aligned16: A, the preconditioner band, b and x are 16-byte aligned (needed
// by the node-pair kernel together with an even n)
// share = 2 (lead) / 3 (partner): the solve takes half of each SM (plan
// kind 4 when it applies), so that two solves on different streams run side
// by side; a lead's CTAs reserve just over half an SM's shared memory, so two
// of them never share an SM, while one partner CTA fits beside each
int pcg_plan(int64_t n, int nf, bool psym_path, bool aligned16, int device, PcgPlan *plan,
             int share = 1);
cudaError_t launch_pcg(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s);
// test hook: 0 = automatic kernel choice, 1 = generic kernel with global
// state, 2 = node-pair kernel with shared-memory state, 3 = node-pair kernel
// with split state, 4 = node-pair kernel with split state on half an SM
// (whenever the forced kind is feasible)
int forced_pcg_kind();
// node-pair kernel (pcg_pair.cu)
size_t pcg_pair_smem(int64_t R);
size_t pcg_pair_split_smem(int64_t R);       // r and p windows only
size_t pcg_pair_split_slice(int64_t R);      // doubles of global workspace per CTA (z/q window)
int pcg_pair_split_occupancy(int mode, size_t smem, int *per_sm);
size_t pcg_pair_half_smem(int64_t R);        // split state at 256 threads
size_t pcg_pair_half_static_smem(int mode);  // the half-SM kernel's static shared memory
int pcg_pair_half_occupancy(int mode, size_t smem, int *per_sm);
int pcg_pair_threads(int kind);   // threads per CTA of plan kind 2, 3 or 4
int pcg_pair_occupancy(int mode, size_t smem, int *per_sm);
cudaError_t launch_pcg_pair(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s);
// batched node-pair kernel: systems `sys`, assignments asg (int4: system,
// group size, rank, rows per CTA) per CTA slot from off[c] to off[c+1].
// half: two lanes of CTA slots, two CTAs per SM (256 threads, half an SM
// each, split state: the z/q window in a per-slot slice of slice_len doubles;
// roles: 2 + 1024 zeroed words) instead of one CTA per SM
int pcg_pair_batch_threads(bool half);
size_t pcg_pair_batch_smem(int64_t R, bool half);
size_t pcg_pair_batch_slice(int64_t R);
size_t pcg_pair_batch_static_smem(bool half);
int pcg_pair_batch_prepare(int mode, size_t smem, bool half);
int pcg_pair_batch_occupancy(int mode, size_t smem, int *per_sm, bool half);
cudaError_t launch_pcg_pair_batch(int mode, int grid, size_t smem, const PcgArgs *sys,
                                  const int4 *asg, const int *off, bool half, unsigned *roles,
                                  double *slices, int slice_len, cudaStream_t s);

}  // namespace airga

namespace airga {
// ---------------------------------------------------------------------------
// host paths for general sparse storage (api_csr.cu)
// ---------------------------------------------------------------------------
int check_any(airga_mat A, const char *name);          // either storage
int csr_check(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
              cudaStream_t s, int32_t *hflag);          // SYNCHRONISES s
int csr_view(airga_mat A, cudaStream_t s, CsrPatPtr *pat, const double **val);
int mat_from_csr_general(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                         const double *val, cudaStream_t s, airga_mat *out);
int assemble_general(airga_mat M, airga_mat K, double alpha, double beta, double sh,
                     cudaStream_t s, airga_mat *A_out);
int spmv_general(airga_mat A, const double *X, double *Y, int32_t m, cudaStream_t s);
int true_residual_general(airga_mat A, const double *X, const double *F, int32_t m,
                          double *relres, cudaStream_t s);
int spai_general(airga_mat A, airga_mat A_old, airga_mat pattern, const airga_options &o,
                 cudaStream_t s, airga_precond_s *out, CsrFactor *F);
int csr_symmetric_part(const CsrFactor &F, cudaStream_t s, CsrFactor *out);
int spai_update_general(airga_precond P_prev, airga_mat A_prev, airga_mat A_next,
                        const airga_options &o, cudaStream_t s, airga_precond_s *P);
int precond_apply_general(airga_precond P, const double *r, double *z, int symmetrize,
                          cudaStream_t s);
int pcg_general(airga_mat A, airga_precond P, const double *F, int32_t m, const airga_options &o,
                double *X, double *res_hist, int32_t *iters, int32_t *status, double *relres,
                int fault, cudaStream_t s);
}  // namespace airga
