// Batched solves: many independent (matrix, preconditioner, right-hand side)
// systems of uneven size in ONE persistent cooperative launch.
//
// Schedule (host, at create): every system gets a group of g CTAs, g chosen
// so that its rows per CTA stay near the requested target and within the
// shared-memory capacity.  Systems are taken in decreasing order of their
// cost estimate (rows, or rows x iterations when the caller supplies costs
// from an earlier run) and each goes to the g CTAs that become free first
// (list scheduling on estimated finish times).  The assignment lists of all
// CTAs follow that single global order, which makes the group barriers
// deadlock free (see pcg_pair_batch_kernel).  Each system has a private
// barrier counter, abort flag, partials block and p boundary buffer.
// With options.sm_share 2 or 3 the CTA slots form two lanes of one slot per
// SM each; a system's group lies within one lane (so its CTAs sit on distinct
// SMs) and each job goes to the lane where it can start first.
//
// The solve call enqueues one memset and one cooperative launch and
// allocates nothing, so it can be captured in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "airga_internal.cuh"

struct airga_batch_s {
    int nsys = 0;
    int grid = 0;
    int mode = 0;
    int64_t rows_target = 0;
    int64_t rows_max = 0;       // largest rows per CTA in the schedule
    size_t smem = 0;
    bool half = false;          // two lanes, two CTAs per SM (options.sm_share 2 or 3)
    double makespan = 0.0;      // estimated, in cost units per CTA
    std::shared_ptr<void> ws;   // device workspace (PcgArgs, assignments, buffers)
    airga::PcgArgs *sys = nullptr;
    int4 *asg = nullptr;
    int *off = nullptr;
    void *ctl = nullptr;
    size_t ctl_bytes = 0;
    unsigned *roles = nullptr;  // lane counters and per-SM arrivals (inside ctl)
    double *slices = nullptr;   // z/q slice per CTA slot (lanes only)
    int slice_len = 0;
};

using namespace airga;

extern "C" {

int airga_batch_create(int32_t nsys, const airga_mat *A, const airga_precond *P,
                       const double *const *F, double *const *X, const double *cost,
                       const int32_t *group, int32_t rows_per_cta, const airga_options *opt,
                       int32_t *iters, int32_t *status, double *relres, void *stream,
                       airga_batch *out) {
    if (!out) return fail(AIRGA_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || !A || !F || !X || !iters || !status || !relres)
        return fail(AIRGA_E_INVALID_ARG, "bad batch arguments");
    airga_options o;
    airga_options_default(&o);
    if (opt) o = *opt;
    int st = check_options(&o);
    if (st) return st;
    int mode = -1;
    for (int s = 0; s < nsys; ++s) {
        st = check_mat(A[s], "A[s]");
        if (st) return st;
        if (A[s]->n % 2 != 0 || !aligned16(F[s]) || !aligned16(X[s]) || !F[s] || !X[s])
            return fail(AIRGA_E_INVALID_ARG, "batch systems need even n and 16-byte aligned F, X");
        const airga_precond p = P ? P[s] : nullptr;
        if (p && (p->n != A[s]->n || p->factors.size() != 1))
            return fail(AIRGA_E_INVALID_ARG, "batch preconditioners must be single factors of matching size");
        const int m_s = p ? 1 : 0;
        if (mode < 0) mode = m_s;
        if (mode != m_s) return fail(AIRGA_E_INVALID_ARG, "all systems need a preconditioner or none");
    }
    int dev = 0, sms = 0, optin = 0, smem_sm = 0, reserved = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    // sm_share 2 or 3: two CTA slots per SM, each with half an SM (the slots
    // of different systems fill each other's barrier gaps)
    const bool half = o.sm_share >= 2;
    const size_t stat = pcg_pair_batch_static_smem(half) + (size_t)reserved;
    // rows per CTA the shared memory can hold
    auto fits = [&](int64_t r) {
        const size_t sm = pcg_pair_batch_smem(r, half);
        return half ? 2 * (sm + stat) <= (size_t)smem_sm && sm + 256 <= (size_t)optin
                    : sm + 512 <= (size_t)optin;
    };
    int64_t rmax = 2;
    while (fits(rmax + 2)) rmax += 2;
    int64_t target = rows_per_cta > 0 ? rows_per_cta : 4096;
    target = std::min<int64_t>(std::max<int64_t>(target, 16), rmax);
    const int G = half ? 2 * sms : sms;          // CTA slots
    const int L = sms;                           // slots per lane (one per SM)
    const int nl = half ? 2 : 1;

    // group sizes
    std::vector<int> g(nsys);
    std::vector<int64_t> R(nsys);
    std::vector<double> c(nsys);
    for (int s = 0; s < nsys; ++s) {
        const int64_t n = A[s]->n;
        int64_t gs = (n + target - 1) / target;
        if (gs < 1) gs = 1;
        if (gs > L) gs = L;                                  // more rows per CTA instead
        if ((n + gs - 1) / gs > rmax) gs = (n + rmax - 1) / rmax;
        if (gs > L) return fail(AIRGA_E_INVALID_ARG, "a batch system is larger than the GPU's shared memory");
        g[s] = (int)gs;
        int64_t rs = (n + gs - 1) / gs;
        rs += rs & 1;
        R[s] = rs;
        c[s] = cost ? std::max(cost[s], 1.0) : (double)n;
    }
    const int64_t rbig = *std::max_element(R.begin(), R.end());
    const size_t smem = pcg_pair_batch_smem(rbig, half);
    // jobs: one system each, or (group given) the systems of one group id with
    // the same group size, placed back to back on one CTA group so that the
    // right-hand sides of one (A, P) reuse its bands while they are in L2
    std::vector<std::vector<int>> jobs;
    if (group) {
        std::vector<std::pair<int64_t, int>> key(nsys);   // (group id, group size) -> job
        std::vector<int> job_of(nsys, -1);
        for (int s = 0; s < nsys; ++s) {
            int found = -1;
            for (int t = 0; t < s && found < 0; ++t)
                if (group[t] == group[s] && g[t] == g[s]) found = job_of[t];
            if (found < 0) {
                found = (int)jobs.size();
                jobs.emplace_back();
            }
            job_of[s] = found;
            jobs[found].push_back(s);
        }
    } else {
        for (int s = 0; s < nsys; ++s) jobs.push_back({s});
    }
    std::vector<double> jc(jobs.size(), 0.0);
    for (size_t j = 0; j < jobs.size(); ++j)
        for (int s : jobs[j]) jc[j] += c[s];
    // list scheduling, largest cost first
    std::vector<int> order(jobs.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jc[a] > jc[b]; });
    std::vector<double> avail(G, 0.0);
    std::vector<std::vector<int4>> lists(G);
    std::vector<int> idx(L), pick(L);
    for (int j : order) {
        const int gj = g[jobs[j][0]];
        double start = 0.0;
        for (int l = 0; l < nl; ++l) {                   // the lane where the job starts first
            std::iota(idx.begin(), idx.end(), l * L);
            std::partial_sort(idx.begin(), idx.begin() + gj, idx.end(), [&](int a, int b) {
                return avail[a] < avail[b] || (avail[a] == avail[b] && a < b);
            });
            double st_l = 0.0;
            for (int k = 0; k < gj; ++k) st_l = std::max(st_l, avail[idx[k]]);
            if (l == 0 || st_l < start) {
                start = st_l;
                std::copy(idx.begin(), idx.begin() + gj, pick.begin());
            }
        }
        std::sort(pick.begin(), pick.begin() + gj);
        const std::vector<int> &sel = pick;
        // members in one global order: every CTA of the group appends them in
        // the same sequence, which keeps the group barriers deadlock free
        for (int s : jobs[j]) {
            const double end = start + c[s] / gj;
            for (int k = 0; k < gj; ++k) lists[sel[k]].push_back(make_int4(s, gj, k, (int)R[s]));
            start = end;
        }
        for (int k = 0; k < gj; ++k) avail[sel[k]] = start;
    }
    const double makespan = *std::max_element(avail.begin(), avail.end());

    // workspace: PcgArgs[nsys] | int4 asg[total] | int off[G+1] | control (2 ints per
    // system; lanes: + 2 + 1024 role counters) | partials (8 g doubles per
    // system) | pbuf (n doubles per system) | lanes: z/q slice per CTA slot
    size_t total_asg = 0;
    for (auto &l : lists) total_asg += l.size();
    size_t nb_pbuf = 0, nb_part = 0;
    for (int s = 0; s < nsys; ++s) {
        nb_pbuf += (size_t)A[s]->n;
        nb_part += (size_t)8 * g[s];
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_sys = al(sizeof(PcgArgs) * nsys), b_asg = al(sizeof(int4) * total_asg),
                 b_off = al(sizeof(int) * (G + 1)), b_bar = al(sizeof(unsigned) * 2 * nsys),
                 b_ctl = b_bar + (half ? al(sizeof(unsigned) * (2 + 1024)) : 0),
                 b_part = al(sizeof(double) * nb_part), b_pbuf = al(sizeof(double) * nb_pbuf);
    const size_t slice_len = pcg_pair_batch_slice(rbig);
    const size_t b_slc = half ? al(sizeof(double) * slice_len * (size_t)G) : 0;
    cudaStream_t cs = (cudaStream_t)stream;
    auto *B = new airga_batch_s;
    st = make_buf(b_sys + b_asg + b_off + b_ctl + b_part + b_pbuf + b_slc, cs, &B->ws);
    if (st) {
        delete B;
        return st;
    }
    char *base = (char *)B->ws.get();
    B->sys = (PcgArgs *)base;
    B->asg = (int4 *)(base + b_sys);
    B->off = (int *)(base + b_sys + b_asg);
    B->ctl = base + b_sys + b_asg + b_off;
    B->ctl_bytes = b_ctl;
    double *part = (double *)(base + b_sys + b_asg + b_off + b_ctl);
    double *pbuf = (double *)(base + b_sys + b_asg + b_off + b_ctl + b_part);
    if (half) {
        B->roles = (unsigned *)((char *)B->ctl + b_bar);
        B->slices = (double *)(base + b_sys + b_asg + b_off + b_ctl + b_part + b_pbuf);
        B->slice_len = (int)slice_len;
    }

    // per-system arguments (host copy, then one upload)
    int32_t *place = placement_buffer();      // test hook: system s records at place[s * 1024 + rank]
    std::vector<PcgArgs> hs(nsys);
    size_t po = 0, pp = 0;
    for (int s = 0; s < nsys; ++s) {
        airga_mat a = A[s];
        if (a->pairz && !a->packed) {
            st = make_buf(sizeof(double) * 5 * (size_t)a->n, cs, &a->packed);
            if (!st) {
                cudaError_t pe = launch_pack_pairs(a->n, a->band->d, (double *)a->packed.get(), cs);
                if (pe != cudaSuccess) st = cuda_fail(pe, "pack pairs");
            }
            if (st) {
                delete B;
                return st;
            }
        }
        PcgArgs &h = hs[s];
        std::memset(&h, 0, sizeof(h));
        h.n = a->n;
        h.A = a->band->d;
        const airga_precond p = P ? P[s] : nullptr;
        h.nf = p ? 1 : 0;
        if (p) {
            h.fac[0] = p->factors[0]->d;
            h.psym = (o.symmetrize && p->psym) ? p->psym->d : nullptr;
        }
        h.symmetrize = o.symmetrize ? 1 : 0;
        h.b = F[s];
        h.x = X[s];
        h.tol = o.tol;
        h.maxit = o.maxit;
        h.warm = o.warm_start ? 1 : 0;
        h.hist = nullptr;
        h.iters = iters + s;
        h.status = status + s;
        h.timeout_ns = (long long)o.barrier_timeout_ms * 1000000ll;
        h.pbuf = pbuf + po;
        h.state = nullptr;
        h.partials = part + pp;
        h.bar = (unsigned *)B->ctl + 2 * s;
        h.abort_flag = (int *)((unsigned *)B->ctl + 2 * s + 1);
        h.fault_skip_arrival = 0;
        h.place = place ? place + (size_t)s * 1024 : nullptr;
        h.pairz = a->pairz ? (const int32_t *)a->pairz.get() : nullptr;
        h.Apk = a->packed ? (const double *)a->packed.get() : nullptr;
        h.relres = relres + s;
        po += (size_t)a->n;
        pp += (size_t)8 * g[s];
    }
    std::vector<int4> hasg;
    std::vector<int> hoff(G + 1, 0);
    for (int k = 0; k < G; ++k) {
        hoff[k] = (int)hasg.size();
        hasg.insert(hasg.end(), lists[k].begin(), lists[k].end());
    }
    hoff[G] = (int)hasg.size();
    cudaError_t e = cudaMemcpyAsync(B->sys, hs.data(), sizeof(PcgArgs) * nsys, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && !hasg.empty())
        e = cudaMemcpyAsync(B->asg, hasg.data(), sizeof(int4) * hasg.size(), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->off, hoff.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);   // host vectors go out of scope
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "batch upload");
    }
    st = pcg_pair_batch_prepare(mode, smem, half);
    if (st) {
        delete B;
        return st;
    }
    int per_sm = 0;
    st = pcg_pair_batch_occupancy(mode, smem, &per_sm, half);
    if (st || per_sm < (half ? 2 : 1)) {
        delete B;
        return st ? st : fail(AIRGA_E_INVALID_ARG, "batch kernel cannot be resident");
    }
    B->half = half;
    B->nsys = nsys;
    B->grid = G;
    B->mode = mode;
    B->rows_target = target;
    B->rows_max = rbig;
    B->smem = smem;
    B->makespan = makespan;
    *out = B;
    return AIRGA_OK;
}

int airga_batch_solve(airga_batch B, void *stream) {
    TraceScope trace_("airga_batch_solve", stream);
    if (!B) return fail(AIRGA_E_INVALID_ARG, "batch is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    AIRGA_CUDA(cudaMemsetAsync(B->ctl, 0, B->ctl_bytes, cs));
    // test hook: an armed fault makes system 0 skip one barrier arrival in
    // this solve only (its flag is set before the launch and cleared after)
    static const int kOne = 1, kZero = 0;
    const bool fault = take_fault(AIRGA_FAULT_SKIP_ARRIVAL);
    int *flag0 = &B->sys[0].fault_skip_arrival;
    if (fault) AIRGA_CUDA(cudaMemcpyAsync(flag0, &kOne, sizeof(int), cudaMemcpyHostToDevice, cs));
    AIRGA_CUDA(launch_pcg_pair_batch(B->mode, B->grid, B->smem, B->sys, B->asg, B->off, B->half,
                                     B->roles, B->slices, B->slice_len, cs));
    if (fault) AIRGA_CUDA(cudaMemcpyAsync(flag0, &kZero, sizeof(int), cudaMemcpyHostToDevice, cs));
    return AIRGA_OK;
}

int airga_batch_info(airga_batch B, int32_t *grid, int32_t *rows_target, int32_t *rows_max,
                     double *makespan) {
    if (!B) return fail(AIRGA_E_INVALID_ARG, "batch is NULL");
    if (grid) *grid = B->grid;
    if (rows_target) *rows_target = (int32_t)B->rows_target;
    if (rows_max) *rows_max = (int32_t)B->rows_max;
    if (makespan) *makespan = B->makespan;
    return AIRGA_OK;
}

void airga_batch_free(airga_batch B) { delete B; }

}  // extern "C"
