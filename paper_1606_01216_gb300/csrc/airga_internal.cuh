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

}  // namespace airga

struct airga_mat_s {
    int64_t n = 0;
    airga::BandPtr band;
    // device int32: nonzero when every row pair (2k, 2k+1) but the last has the
    // Hermite-beam zeros (even rows: offsets -3, +1; odd rows: +3, -1)
    std::shared_ptr<void> pairz;
    // packed copy of the beam's nonzero entries for the PCG row-pair stencil
    // (5 doubles per row, made on the first solve with this matrix)
    std::shared_ptr<void> packed;
};

struct airga_precond_s {
    int64_t n = 0;
    std::vector<airga::BandPtr> factors;  // factor 0 = built P, then Q_2, Q_3, ...
    airga::BandPtr psym;                  // 1/2 (P + P^T) when factors.size() == 1
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

// ---------------------------------------------------------------------------
// persistent PCG (pcg_kernel.cu)
// ---------------------------------------------------------------------------
constexpr int kMaxChain = 16;

struct PcgPlan {
    int kind = 0;          // 0 generic (shared-memory state), 1 generic (global state), 2 node-pair,
                           // 3 node-pair with r, p in shared memory and x, z/q in global memory
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
};

// process-wide test fault consumed by the next pcg_solve (airga_debug_set_fault)
int take_fault();

// aligned16: A, the preconditioner band, b and x are 16-byte aligned (needed
// by the node-pair kernel together with an even n)
int pcg_plan(int64_t n, int nf, bool psym_path, bool aligned16, int device, PcgPlan *plan);
cudaError_t launch_pcg(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s);
// test hook: 0 = automatic kernel choice, 1 = generic kernel with global
// state, 2 = node-pair kernel with shared-memory state, 3 = node-pair kernel
// with split state (whenever the forced kind is feasible)
int forced_pcg_kind();
// node-pair kernel (pcg_pair.cu)
size_t pcg_pair_smem(int64_t R);
size_t pcg_pair_split_smem(int64_t R);       // r and p windows only
size_t pcg_pair_split_slice(int64_t R);      // doubles of global workspace per CTA (z/q window)
int pcg_pair_split_occupancy(int mode, size_t smem, int *per_sm);
int pcg_pair_threads(int kind);   // threads per CTA of plan kind 2 or 3
int pcg_pair_occupancy(int mode, size_t smem, int *per_sm);
cudaError_t launch_pcg_pair(const PcgPlan &plan, const PcgArgs &args, cudaStream_t s);
// batched node-pair kernel: systems `sys`, assignments asg (int4: system,
// group size, rank, rows per CTA) per CTA from off[c] to off[c+1]
int pcg_pair_batch_prepare(int mode, size_t smem);
int pcg_pair_batch_occupancy(int mode, size_t smem, int *per_sm);
cudaError_t launch_pcg_pair_batch(int mode, int grid, size_t smem, const PcgArgs *sys,
                                  const int4 *asg, const int *off, cudaStream_t s);

}  // namespace airga
