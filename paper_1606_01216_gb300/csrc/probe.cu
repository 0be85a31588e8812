// Measurement aid (no counterpart in the paper): the FP64 FMA issue rate of
// the device, the roofline of the FP64-bound kernels of this library (PCG,
// SPAI QR, MR).  One CTA of 1024 threads per SM (the dynamic shared-memory
// request keeps a second CTA off the SM), each thread running 8, 12 or 16
// independent FMA chains (the best of the three counts); the SM's own cycle
// counter brackets the chains, so the result
// is FMAs per SM clock, independent of the clock the GPU runs at.  The event
// time of the launch gives the TFLOP/s at the clocks of the moment.
#include <algorithm>
#include <vector>

#include "airga_internal.cuh"

namespace airga {
namespace {

constexpr int kProbeThreads = 1024;

// CHAINS independent FMA chains per thread, 4 steps per loop trip (a 32-bit
// trip counter), so loop overhead stays far below the FP64 issue rate.
template <int CHAINS>
__global__ void __launch_bounds__(kProbeThreads, 1)
fp64_rate_kernel(int trips, double seed, double mul, double add, double *sink,
                 long long *cycles) {
    extern __shared__ double pad[];
    double a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = seed + 1e-9 * threadIdx.x + c;
    __syncthreads();
    const long long t0 = clock64();
    for (int k = 0; k < trips; ++k) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], mul, add);
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == 0.125) sink[threadIdx.x] = s + pad[0];   // keeps the chains live, never true
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace airga

using namespace airga;

extern "C" int airga_probe_fp64_rate(int64_t iters, double *fma_per_clk_sm, double *tflops,
                                     double *ms, void *stream) {
    if (iters < 1 || iters > (int64_t)1 << 24)
        return fail(AIRGA_E_INVALID_ARG, "iters must be in [1, 2^24]");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, smem_sm = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    AIRGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AIRGA_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const size_t smem = (size_t)smem_sm / 2 + 1024;   // a second CTA cannot fit
    void *buf = nullptr;
    int st = dev_alloc(&buf, sizeof(long long) * sms + sizeof(double) * kProbeThreads, s);
    if (st) return st;
    long long *cyc = (long long *)buf;
    double *sink = (double *)(cyc + sms);
    cudaEvent_t e0, e1;
    AIRGA_CUDA(cudaEventCreate(&e0));
    AIRGA_CUDA(cudaEventCreate(&e1));
    std::vector<long long> h(sms);
    const int trips = (int)((iters + 3) / 4);
    double best_rate = 0.0, best_tf = 0.0, best_ms = 0.0;
    cudaError_t e = cudaSuccess;
    // 8, 12 and 16 chains per thread (more would spill at 64 registers): the
    // best of the three is the rate
    for (int variant = 0; variant < 3 && e == cudaSuccess; ++variant) {
        const int chains = 8 + 4 * variant;
        const void *kern = variant == 0 ? (const void *)fp64_rate_kernel<8>
                         : variant == 1 ? (const void *)fp64_rate_kernel<12>
                                        : (const void *)fp64_rate_kernel<16>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) break;
        double seed = 1.0, mul = 1.0 - 1e-12, add = 1e-13;   // the chains stay bounded
        int tr = trips;
        void *args[] = {(void *)&tr, (void *)&seed, (void *)&mul, (void *)&add, (void *)&sink,
                        (void *)&cyc};
        float t = 0.f;
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = cudaLaunchKernel(kern, dim3(sms), dim3(kProbeThreads), args, smem, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) break;
        std::sort(h.begin(), h.end());
        const double fmas_cta = (double)kProbeThreads * chains * 4.0 * (double)trips;
        const double med = (double)h[h.size() / 2];
        const double rate = med > 0 ? fmas_cta / med : 0.0;
        if (rate > best_rate) {
            best_rate = rate;
            best_tf = t > 0 ? 2.0 * fmas_cta * sms / (t * 1e-3) / 1e12 : 0.0;
            best_ms = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 rate probe");
    if (fma_per_clk_sm) *fma_per_clk_sm = best_rate;
    if (tflops) *tflops = best_tf;
    if (ms) *ms = best_ms;
    return AIRGA_OK;
}

// ---------------------------------------------------------------------------
// Read bandwidth of a buffer of `bytes` (no counterpart in the paper): a
// buffer below the L2 size measures L2 read bandwidth, a larger one DRAM.
// Every thread streams 16-byte loads that bypass L1 (ld.global.cg) in a
// grid-stride loop; one untimed pass warms the cache, then `passes` passes
// are timed with events.  The XOR of everything read goes to `sink` only if
// it has an impossible value, so the loads cannot be removed.
// ---------------------------------------------------------------------------
namespace airga {
namespace {

__global__ void __launch_bounds__(512)
read_bw_kernel(const uint4 *__restrict__ buf, int64_t n16, int passes, unsigned *sink) {
    unsigned acc = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

}  // namespace
}  // namespace airga

extern "C" int airga_probe_read_bw(int64_t bytes, int32_t passes, double *gbs, double *ms,
                                   void *stream) {
    if (bytes < (1 << 20) || bytes > ((int64_t)16 << 30) || (bytes & 15))
        return fail(AIRGA_E_INVALID_ARG, "bytes must be a multiple of 16 in [1 MiB, 16 GiB]");
    if (passes < 1 || passes > 1000) return fail(AIRGA_E_INVALID_ARG, "passes must be in [1, 1000]");
    if (!gbs) return fail(AIRGA_E_INVALID_ARG, "gbs is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    AIRGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    void *buf = nullptr;
    int st = dev_alloc(&buf, (size_t)bytes + 64, s);
    if (st) return st;
    unsigned *sink = (unsigned *)((char *)buf + bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(buf, 0x5A, (size_t)bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int64_t n16 = bytes / 16;
    const unsigned grid = (unsigned)sms * 4u;
    float t = 0.f;
    if (e == cudaSuccess) {
        read_bw_kernel<<<grid, 512, 0, s>>>((const uint4 *)buf, n16, 1, sink);   // warm
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        read_bw_kernel<<<grid, 512, 0, s>>>((const uint4 *)buf, n16, passes, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "read bandwidth probe");
    *gbs = t > 0.f ? (double)bytes * passes / (t * 1e-3) / 1e9 : 0.0;
    if (ms) *ms = t;
    return AIRGA_OK;
}
