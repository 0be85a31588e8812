// airga_pcg_solve_noalloc: the persistent PCG of airga_pcg_solve for callers
// that cannot let a library allocate device memory.
//
// Who needs it: an application whose device memory is owned end to end by its
// own allocator (for example a framework that reserves the whole GPU up front
// and forbids libraries from allocating behind its back), and latency-critical
// loops that cannot afford the synchronisation or the failure point an
// allocation call brings.  Such a caller passes every input and output buffer
// itself; the only other memory this entry point touches is the fixed scratch
// array below, which exists for the whole life of the process on every GPU
// that loads the library.
//
// Scratch contents (doubles): the boundary rows of p (up to kNoallocMaxRows),
// the per-CTA z/q window slices of the split-state plan (even n whose four
// shared-memory windows no longer fit, from about 1.04e6 rows on 152 SMs),
// the per-CTA reduction partials, the partials of the true residual and the
// barrier control words.  Every call reuses the same array and it keeps the
// previous call's contents, so the control words are cleared on the stream
// before each column; calls whose work overlaps on the GPU (concurrent
// streams, other threads) race on the array and must be serialised by the
// caller.
#include <mutex>

#include "airga_internal.cuh"

namespace airga {
namespace {

constexpr int64_t kNoallocMaxRows = 1 << 20;                  // 1,048,576 rows
constexpr int64_t kNoallocMaxCtas = 1024;
constexpr int64_t kNoallocResidBlocks = 1216;
constexpr int64_t kNoallocPbuf = kNoallocMaxRows;
// split-state slices: (R + 8) doubles per CTA with R <= n / grid + 2
constexpr int64_t kNoallocSlices = kNoallocMaxRows + 16 * kNoallocMaxCtas;
constexpr int64_t kNoallocPartials = 2 * 4 * kNoallocMaxCtas;
constexpr int64_t kNoallocResid = 2 * kNoallocResidBlocks;
constexpr int64_t kNoallocCtl = 32;                           // barrier counter + abort flag, padded
constexpr int64_t kNoallocDoubles =
    kNoallocPbuf + kNoallocSlices + kNoallocPartials + kNoallocResid + kNoallocCtl;

// 16.2 MiB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[128] = {};   // device address of the array, per device ordinal

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
int noalloc_scratch(double **out) {
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(AIRGA_E_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return AIRGA_OK;
}

}  // namespace
}  // namespace airga

using namespace airga;

extern "C" int airga_pcg_solve_noalloc(int64_t n, const double *A_band, const double *M_band,
                                       const double *F, int32_t m, const airga_options *opt,
                                       double *X, double *res_hist, int32_t *iters,
                                       int32_t *status, double *true_relres, void *stream) {
    if (n < 1) return fail(AIRGA_E_INVALID_ARG, "n must be >= 1");
    if (n > kNoallocMaxRows)
        return fail(AIRGA_E_INVALID_ARG,
                    "pcg_solve_noalloc: n exceeds the fixed scratch capacity of 1048576 rows");
    if (m < 0) return fail(AIRGA_E_INVALID_ARG, "m must be >= 0");
    if (m == 0) return AIRGA_OK;
    if (!A_band || !F || !X || !iters || !status || !true_relres)
        return fail(AIRGA_E_INVALID_ARG, "A_band, F, X, iters, status and true_relres are required");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    if (!(o.tol >= 0.0) || o.maxit < 0 || o.barrier_timeout_ms <= 0)
        return fail(AIRGA_E_INVALID_ARG, "bad tol, maxit or barrier_timeout_ms");

    double *scratch = nullptr;
    int st = noalloc_scratch(&scratch);
    if (st) return st;
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    const int nf = M_band ? 1 : 0;
    const bool al = ((uintptr_t)A_band & 15u) == 0 && ((uintptr_t)F & 15u) == 0 &&
                    ((uintptr_t)X & 15u) == 0 && ((uintptr_t)M_band & 15u) == 0;
    PcgPlan plan;
    st = pcg_plan(n, nf, false, al, dev, &plan);
    if (st) return st;
    // every plan but the generic kernel with its whole state in global memory
    // (kind 1) fits: shared-memory state, or the split state whose z/q slices
    // live in the array
    if (plan.kind == 1 || (int64_t)plan.scratch_doubles > kNoallocSlices)
        return fail(AIRGA_E_INVALID_ARG,
                    "pcg_solve_noalloc: the solve state does not fit in shared memory on this GPU");
    if (plan.grid > kNoallocMaxCtas)
        return fail(AIRGA_E_INVALID_ARG, "pcg_solve_noalloc: grid larger than the scratch allows");
    const int nblk = true_residual_blocks(n);
    if (nblk > kNoallocResidBlocks)
        return fail(AIRGA_E_INVALID_ARG, "pcg_solve_noalloc: residual blocks exceed the scratch");

    cudaStream_t s = (cudaStream_t)stream;
    PcgArgs a{};
    a.n = n;
    a.A = A_band;
    a.nf = nf;
    // the caller's band is applied as given, z = M r, by every kernel variant:
    // a plain factor read through all seven diagonals, no symmetry assumed
    a.fac[0] = M_band;
    a.psym = nullptr;
    a.symmetrize = 0;
    a.tol = o.tol;
    a.maxit = o.maxit;
    a.warm = o.warm_start ? 1 : 0;
    a.timeout_ns = (long long)o.barrier_timeout_ms * 1000000ll;
    a.fault_skip_arrival = 0;
    a.pbuf = scratch;
    a.state = plan.scratch_doubles ? scratch + kNoallocPbuf : nullptr;
    a.partials = scratch + kNoallocPbuf + kNoallocSlices;
    double *resid = a.partials + kNoallocPartials;
    unsigned *ctl = (unsigned *)(resid + kNoallocResid);
    a.bar = ctl;
    a.abort_flag = (int *)(ctl + 1);
    cudaError_t e = cudaSuccess;
    for (int32_t c = 0; c < m && e == cudaSuccess; ++c) {
        a.b = F + (size_t)c * n;
        a.x = X + (size_t)c * n;
        a.hist = res_hist ? res_hist + (size_t)c * (o.maxit + 1) : nullptr;
        a.iters = iters + c;
        a.status = status + c;
        e = cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess) e = launch_pcg(plan, a, s);
        if (e == cudaSuccess)
            e = launch_true_residual(n, A_band, a.x, a.b, 1, true_relres + c, resid, nblk, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pcg_solve_noalloc launch");
    return AIRGA_OK;
}
