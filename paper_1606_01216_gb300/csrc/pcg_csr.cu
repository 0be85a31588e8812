// Persistent preconditioned CG for matrices in general sparse (CSR)
// storage: the same Hestenes-Stiefel recurrence as the band kernels (the CG
// solves of Alg. 3 line 5, Alg. 5 lines 7/11), with A and the preconditioner
// factors read through row views and every vector in global memory.
//
// One cooperative launch per right-hand side; thread t of the grid owns rows
// t, t + T, t + 2T, ... for the whole solve.  A CSR row may reach any other
// row, so vectors are exchanged through global memory (L2) at grid barriers:
//   B0  after p = z + beta p                -> p visible to all
//   B1  after q = A p and (p, q)            -> alpha
//   B2  after x += alpha p, r -= alpha q    -> ||r||, r visible to all
//       [one barrier per further factor of an update chain]
//   B3  after z = M r and (r, z)            -> beta, z visible to all
// (Forming p_c = z_c + beta p_c inside q's gather instead of exchanging p
// saves B0 but doubles the gathers and adds an FMA per entry; with two CTAs
// per SM the barrier is the cheaper of the two.)  The previous and the new p
// live in two buffers (iteration parity).
#include <cstring>

#include "csr_common.cuh"
#include "pcg_common.cuh"

namespace airga {
namespace {

using namespace pcgdev;

constexpr int kThreads = 256;

struct CsrPcgArgs {
    int64_t n;
    RowView A;
    int nf;                      // chain length, 0 = identity
    RowView fwd[kMaxChain];      // factor k
    RowView tr[kMaxChain];       // factor k transposed
    RowView sym;                 // symmetric part of a single factor
    int use_sym;
    int symmetrize;
    const double *b;
    double *x;
    double tol;
    int maxit;
    int warm;
    double *hist;
    int32_t *iters;
    int32_t *status;
    double *relres;
    long long timeout_ns;
    double *r, *z, *q, *p[2], *t[2], *u[2];
    double *partials;
    unsigned *bar;
    int *abort_flag;
    int fault_skip_arrival;
};

// z = M r on own rows (chain stages exchange through global memory)
__device__ __forceinline__ bool apply_M(const CsrPcgArgs &a, int64_t g0, int64_t gs,
                                        unsigned &bar_no, int G, int *s_flag) {
    const int64_t n = a.n;
    if (a.use_sym) {
        for (int64_t i = g0; i < n; i += gs) a.z[i] = rv_dot_cg(a.sym, i, a.r);
        return true;
    }
    if (a.nf == 0) {
        for (int64_t i = g0; i < n; i += gs) a.z[i] = a.r[i];
        return true;
    }
    // C r = F_{nf-1} ... F_0 r and C^T r = F_0^T ... F_{nf-1}^T r, stage by stage
    const double *st = a.r, *su = a.r;
    for (int s = 0; s < a.nf; ++s) {
        double *dt = (s & 1) ? a.t[1] : a.t[0], *du = (s & 1) ? a.u[1] : a.u[0];
        for (int64_t i = g0; i < n; i += gs) {
            dt[i] = rv_dot_cg(a.fwd[s], i, st);
            if (a.symmetrize) du[i] = rv_dot_cg(a.tr[a.nf - 1 - s], i, su);
        }
        st = dt;
        su = du;
        if (s + 1 < a.nf) {
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, a.timeout_ns, s_flag))
                return false;
            ++bar_no;
        }
    }
    for (int64_t i = g0; i < n; i += gs)
        a.z[i] = a.symmetrize ? 0.5 * (__ldcg(st + i) + __ldcg(su + i)) : __ldcg(st + i);
    return true;
}

__global__ void __launch_bounds__(kThreads) pcg_csr_kernel(CsrPcgArgs a) {
    __shared__ double red[160];
    __shared__ int s_flag;
    const int G = gridDim.x;
    const int64_t n = a.n;
    const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t gs = (int64_t)gridDim.x * blockDim.x;
    const long long tmo = a.timeout_ns;
    unsigned bar_no = 0;
    int status = AIRGA_E_MAXIT;
    int iters = 0;
    double nb = 0.0;

    // ---- x_0, r_0 = b - A x_0 ----
    {
        double v[1] = {0.0};
        for (int64_t i = g0; i < n; i += gs) {
            const double bi = a.b[i];
            double ri = bi;
            if (a.warm) ri = bi - rv_dot(a.A, i, a.x);
            else a.x[i] = 0.0;
            a.r[i] = ri;
            v[0] = fma(bi, bi, v[0]);
        }
        block_partials<1>(v, red, a.partials, bar_no & 1, G);
    }
    if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
        status = AIRGA_E_TIMEOUT;
        goto finish;
    }
    {
        double t[1];
        grid_totals<1>(a.partials, bar_no & 1, G, red + 128, t);
        ++bar_no;
        nb = sqrt(t[0]);
    }
    if (nb == 0.0) {
        for (int64_t i = g0; i < n; i += gs) a.x[i] = 0.0;
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[0] = 0.0;
        status = AIRGA_OK;
        goto finish;
    }
    if (!apply_M(a, g0, gs, bar_no, G, &s_flag)) {
        status = AIRGA_E_TIMEOUT;
        goto finish;
    }
    {
        double v[2] = {0.0, 0.0};
        for (int64_t i = g0; i < n; i += gs) {
            const double ri = a.r[i];
            v[0] = fma(ri, a.z[i], v[0]);
            v[1] = fma(ri, ri, v[1]);
        }
        block_partials<2>(v, red, a.partials, bar_no & 1, G);
    }
    if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
        status = AIRGA_E_TIMEOUT;
        goto finish;
    }
    {
        double t0[2];
        grid_totals<2>(a.partials, bar_no & 1, G, red + 128, t0);
        ++bar_no;
        double rz = t0[0];
        double rn = sqrt(t0[1]);
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[0] = rn / nb;
        if (rn <= a.tol * nb) { status = AIRGA_OK; goto finish; }
        if (!isfinite(rz) || rz == 0.0) { status = AIRGA_E_BREAKDOWN; goto finish; }
        double beta = 0.0;
        for (int k = 1; k <= a.maxit; ++k) {
            double *pc = (k & 1) ? a.p[1] : a.p[0];
            const double *pp = (k & 1) ? a.p[0] : a.p[1];
            // ---- p = z + beta p_prev on own rows, exchanged at a barrier ----
            for (int64_t i = g0; i < n; i += gs) pc[i] = k == 1 ? a.z[i] : fma(beta, pp[i], a.z[i]);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
                status = AIRGA_E_TIMEOUT;
                iters = k - 1;
                goto finish;
            }
            ++bar_no;
            // ---- q = A p, (p, q) ----
            double vq[1] = {0.0};
            for (int64_t i = g0; i < n; i += gs) {
                int64_t rb, re;
                rv_range(a.A, i, rb, re);
                double acc = 0.0;
                for (int64_t e = rb; e < re; ++e) {
                    const int64_t c = rv_col(a.A, e);
                    if (c < 0) continue;
                    acc = fma(rv_val(a.A, e), __ldcg(pc + c), acc);
                }
                const double pi = pc[i];
                a.q[i] = acc;
                vq[0] = fma(pi, acc, vq[0]);
            }
            block_partials<1>(vq, red, a.partials, bar_no & 1, G);
            const bool arrive = !(a.fault_skip_arrival && k == 1 && blockIdx.x == 0);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag, arrive)) {
                status = AIRGA_E_TIMEOUT;
                iters = k - 1;
                goto finish;
            }
            double pqt[1];
            grid_totals<1>(a.partials, bar_no & 1, G, red + 128, pqt);
            ++bar_no;
            const double pq = pqt[0];
            if (!(pq > 0.0) || !isfinite(pq)) {
                status = AIRGA_E_BREAKDOWN;
                iters = k - 1;
                goto finish;
            }
            const double alpha = rz / pq;
            // ---- x += alpha p, r -= alpha q ----
            double vr[1] = {0.0};
            for (int64_t i = g0; i < n; i += gs) {
                a.x[i] = fma(alpha, pc[i], a.x[i]);
                const double ri = fma(-alpha, a.q[i], a.r[i]);
                a.r[i] = ri;
                vr[0] = fma(ri, ri, vr[0]);
            }
            block_partials<1>(vr, red, a.partials, bar_no & 1, G);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
                status = AIRGA_E_TIMEOUT;
                iters = k;
                goto finish;
            }
            double rrt[1];
            grid_totals<1>(a.partials, bar_no & 1, G, red + 128, rrt);
            ++bar_no;
            iters = k;
            rn = sqrt(rrt[0]);
            if (blockIdx.x == 0 && threadIdx.x == 0 && a.hist) a.hist[k] = rn / nb;
            if (rn <= a.tol * nb) { status = AIRGA_OK; break; }
            // ---- z = M r, (r, z) ----
            if (!apply_M(a, g0, gs, bar_no, G, &s_flag)) {
                status = AIRGA_E_TIMEOUT;
                goto finish;
            }
            double vz[1] = {0.0};
            for (int64_t i = g0; i < n; i += gs) vz[0] = fma(a.r[i], a.z[i], vz[0]);
            block_partials<1>(vz, red, a.partials, bar_no & 1, G);
            if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) {
                status = AIRGA_E_TIMEOUT;
                goto finish;
            }
            double rzt[1];
            grid_totals<1>(a.partials, bar_no & 1, G, red + 128, rzt);
            ++bar_no;
            const double rz_new = rzt[0];
            if (!isfinite(rz_new) || rz_new == 0.0) { status = AIRGA_E_BREAKDOWN; break; }
            beta = rz_new / rz;
            rz = rz_new;
        }
    }
finish:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.iters = iters;
        *a.status = status;
    }
    if (a.relres) {
        if (status == AIRGA_E_TIMEOUT) {
            if (blockIdx.x == 0 && threadIdx.x == 0)
                *a.relres = __longlong_as_double(0x7FF8000000000000ll);   // no residual pass
            return;
        }
        // true residual ||b - A x|| / ||b|| of the final x (x exchanged at one barrier)
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) return;
        ++bar_no;
        double v[2] = {0.0, 0.0};
        for (int64_t i = g0; i < n; i += gs) {
            const double bi = a.b[i], ri = bi - rv_dot_cg(a.A, i, a.x);
            v[0] = fma(ri, ri, v[0]);
            v[1] = fma(bi, bi, v[1]);
        }
        block_partials<2>(v, red, a.partials, bar_no & 1, G);
        if (!grid_barrier(a.bar, a.abort_flag, (bar_no + 1) * (unsigned)G, tmo, &s_flag)) return;
        double t[2];
        grid_totals<2>(a.partials, bar_no & 1, G, red + 128, t);
        if (blockIdx.x == 0 && threadIdx.x == 0) *a.relres = t[1] > 0.0 ? sqrt(t[0]) / sqrt(t[1]) : 0.0;
    }
}

}  // namespace

// Workspace: 9 n doubles of vectors, partials and the control words.
size_t pcg_csr_workspace_doubles(int64_t n, int grid) {
    return (size_t)9 * (size_t)n + (size_t)8 * (size_t)grid + 8;
}

int pcg_csr_grid(int64_t n, int device, int *grid) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_csr_kernel, kThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pcg csr occupancy");
    if (per_sm < 1) return fail(AIRGA_E_CUDA, "pcg csr: kernel cannot be resident");
    int64_t want = (n + kThreads - 1) / kThreads;
    // two CTAs per SM at most: fewer partials and barrier arrivals per grid
    // reduction (91 us per iteration on a 490,700-row membrane against 95 at
    // four per SM and 98 at full occupancy)
    int64_t cap = (int64_t)(per_sm < 2 ? per_sm : 2) * sms;
    *grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    return AIRGA_OK;
}

// One solve per column of F.  ws: pcg_csr_workspace_doubles(n, grid) doubles,
// control words (2 unsigned) at its end, zeroed here before each column.
int launch_pcg_csr(int64_t n, int grid, const RowView &A, int nf, const RowView *fwd,
                   const RowView *tr, const RowView *sym, int symmetrize, const double *F,
                   int32_t m, double *X, double *res_hist, int32_t maxit, double tol, int warm,
                   long long timeout_ns, int fault, int32_t *iters, int32_t *status,
                   double *relres, double *ws, cudaStream_t s) {
    CsrPcgArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.A = A;
    a.nf = nf;
    for (int k = 0; k < nf; ++k) {
        a.fwd[k] = fwd[k];
        a.tr[k] = tr[k];
    }
    a.use_sym = sym ? 1 : 0;
    if (sym) a.sym = *sym;
    a.symmetrize = symmetrize;
    a.tol = tol;
    a.maxit = maxit;
    a.warm = warm;
    a.timeout_ns = timeout_ns;
    double *v = ws;
    a.r = v; v += n;
    a.z = v; v += n;
    a.q = v; v += n;
    a.p[0] = v; v += n;
    a.p[1] = v; v += n;
    a.t[0] = v; v += n;
    a.t[1] = v; v += n;
    a.u[0] = v; v += n;
    a.u[1] = v; v += n;
    a.partials = v; v += (size_t)8 * grid;
    unsigned *ctl = (unsigned *)v;
    a.bar = ctl;
    a.abort_flag = (int *)(ctl + 1);
    for (int32_t c = 0; c < m; ++c) {
        a.b = F + (size_t)c * n;
        a.x = X + (size_t)c * n;
        a.hist = res_hist ? res_hist + (size_t)c * (maxit + 1) : nullptr;
        a.iters = iters + c;
        a.status = status + c;
        a.relres = relres + c;
        a.fault_skip_arrival = (fault && c == 0) ? 1 : 0;
        cudaError_t e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess) e = injected_launch_error();   // host-side test fault only
        if (e == cudaSuccess) {
            void *kargs[] = {(void *)&a};
            e = cudaLaunchCooperativeKernel((const void *)pcg_csr_kernel, dim3(grid), dim3(kThreads),
                                            kargs, 0, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "pcg csr launch");
    }
    return AIRGA_OK;
}

}  // namespace airga

AIRGA_CHECK_READER(pcg_csr)
