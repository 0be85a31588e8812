// Device helpers shared by the persistent PCG kernels: bounded grid barrier,
// deterministic block and grid reductions.
#pragma once

#include "airga_internal.cuh"

namespace airga {
namespace pcgdev {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier.  Returns false (in every thread) if this CTA gave up.
// `arrive` is false only under the test fault injection (a CTA that never
// arrives, so every wait runs into its bound).
// `grid_size` 1 (a group of one CTA; 0 = not stated): the CTA barrier alone
// orders the CTA's writes before its own later reads, so the counter round
// trip is skipped (unless the test fault withholds the arrival).
__device__ bool grid_barrier(unsigned *bar, int *abort_flag, unsigned target,
                             long long timeout_ns, int *s_flag, bool arrive = true,
                             int grid_size = 0) {
    __syncthreads();
    if (grid_size == 1 && arrive) return true;
    if (threadIdx.x == 0) {
        // release-reduction: orders this CTA's writes (gathered by the CTA
        // barrier above) before the arrival, without a separate fence
        if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        int ok = 1;
        unsigned long long t0 = global_ns();
        // bounded by the timer and, should the timer stall, by a poll count
        // (each poll is an L2 round trip, far longer than 16 ns)
        const unsigned long long max_spins = (unsigned long long)(timeout_ns > 0 ? timeout_ns : 0) / 16 + 64;
        unsigned long long spins = 0;
        while (ld_acquire(bar) < target) {
            if ((++spins & 63u) == 0) {
                if (*(volatile int *)abort_flag) { ok = 0; break; }
                if ((long long)(global_ns() - t0) > timeout_ns || spins > max_spins) {
                    atomicExch(abort_flag, 1);
                    ok = 0;
                    break;
                }
            }
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-sum NV values; thread 0 writes them to partials[slot][v][cta].
template <int NV>
__device__ void block_partials(double (&v)[NV], double *red, double *partials, int slot,
                               int grid) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q * 32 + w] = v[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double t = l < nw ? red[q * 32 + l] : 0.0;
            t = warp_sum(t);
            if (l == 0) partials[(slot * 4 + q) * grid + blockIdx.x] = t;
        }
    }
}

// After a barrier: every CTA sums the G partials of `slot` in the same order;
// the NV totals go through the shared slots `out_sm` to every thread.
template <int NV>
__device__ void grid_totals(const double *partials, int slot, int grid, double *out_sm,
                            double (&out)[NV]) {
    // warp q sums value q: the NV sums run side by side.  Every lane issues
    // all of its loads before the first add, so the partials (written by
    // other SMs, read from L2) cost one round trip instead of one per add.
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < NV) {
        const double *src = partials + (slot * 4 + w) * grid;
        constexpr int kPerLane = 8;                 // up to 256 CTAs in one sweep
        double v[kPerLane];
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            const int g = l + 32 * j;
            v[j] = g < grid ? __ldcg(src + g) : 0.0;
        }
        double t = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
        for (int g = l + 32 * kPerLane; g < grid; g += 32) t += __ldcg(src + g);
        t = warp_sum(t);
        if (l == 0) out_sm[w] = t;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = out_sm[q];
    __syncthreads();
}

// Warp 0 alone sums the NV partials of `slot` (all lanes' loads issued
// together, fixed order, identical in every CTA) into tot[0..NV); call from
// warp 0 only, then derive the scalars there and broadcast them through
// shared memory.  Keeping the scalar FP64 work (divisions, tests) in one
// warp matters on GB300, where each warp-wide FP64 instruction occupies the
// FP64 pipe of its SM sub-partition for ~64 cycles.
template <int NV>
__device__ __forceinline__ void warp0_totals(const double *partials, int slot, int grid,
                                             double (&tot)[NV]) {
    const int l = threadIdx.x & 31;
    constexpr int kPerLane = 8;                     // up to 256 CTAs in one sweep
    double v[NV][kPerLane];
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int j = 0; j < kPerLane; ++j) {
            const int g = l + 32 * j;
            v[q][j] = g < grid ? __ldcg(partials + (slot * 4 + q) * grid + g) : 0.0;
        }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = ((v[q][0] + v[q][1]) + (v[q][2] + v[q][3])) +
                   ((v[q][4] + v[q][5]) + (v[q][6] + v[q][7]));
        for (int g = l + 32 * kPerLane; g < grid; g += 32)
            t += __ldcg(partials + (slot * 4 + q) * grid + g);
        tot[q] = warp_sum(t);
    }
}

// Block-sum NV values with a shared-memory tree; thread 0 writes them to
// partials[slot][v][cta].  `red` holds NV * blockDim.x doubles.  On GB300 a
// warp-wide FP64 add occupies the FP64 pipe for ~64 cycles, so the tree
// halves the number of participating warps at each level instead of running
// a 5-level shuffle tree in every warp (about 20 warp-wide adds per value
// instead of 85 for 512 threads).  blockDim.x must be a multiple of 128.
template <int NV>
__device__ void block_partials_tree(double (&v)[NV], double *red, double *partials, int slot,
                                    int grid, int rank) {
    const int tid = threadIdx.x, nt = blockDim.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) red[q * nt + tid] = v[q];
    __syncthreads();
    const int quarter = nt >> 2;
    if (tid < quarter) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double *r = red + q * nt;
            r[tid] = (r[tid] + r[tid + quarter]) + (r[tid + 2 * quarter] + r[tid + 3 * quarter]);
        }
    }
    __syncthreads();
    const int w = tid >> 5, l = tid & 31;
    if (w < NV) {                      // warp q finishes value q
        const double *r = red + w * nt;
        double t;
        if (quarter == 128) {          // 512 threads: four values per lane, loaded together
            const double a0 = r[l], a1 = r[l + 32], a2 = r[l + 64], a3 = r[l + 96];
            t = (a0 + a1) + (a2 + a3);
        } else {
            t = 0.0;
            for (int k = l; k < quarter; k += 32) t += r[k];
        }
        t = warp_sum(t);
        if (l == 0) partials[(slot * 4 + w) * grid + rank] = t;
    }
}

}  // namespace
}  // namespace pcgdev
}  // namespace airga
