// tcgen05 building blocks (sm_100-family tensor cores): shared-memory matrix
// descriptors, BF16 MMA into tensor memory, commit / bounded mbarrier wait,
// tensor-memory loads.  Operands live in shared memory in the no-swizzle
// K-major "core matrix" layout: 8 rows x 16 bytes per core matrix, core
// matrices adjacent in K are 128 bytes apart (leading-dimension offset),
// those adjacent in M/N are (K/8)*128 bytes apart (stride-dimension offset).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace airga {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of an operand with K columns
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int K) {
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void st_bf16(uint8_t *base, int r, int k, int K, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + kmaj_off(r, k, K)) = __float2bfloat16(v);
}

__device__ __forceinline__ float ld_bf16(const uint8_t *base, int r, int k, int K) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(base + kmaj_off(r, k, K)));
}

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version bits (0b001); no swizzle, base offset 0
    return d;
}

// kind::f16 instruction descriptor: BF16 A and B (K-major), FP32 D, M x N
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D[128 x N] (+)= A[128 x K] * B[N x K]^T, operands in shared memory with K
// columns each; issued by ONE thread.  K a multiple of 16.
__device__ __forceinline__ void gemm(uint32_t tmem_d, const uint8_t *A, const uint8_t *B, int K,
                                     int N, bool accumulate) {
    const uint32_t sbo = (uint32_t)(K >> 3) * 128;
    const uint32_t id = idesc_bf16(128, N);
    for (int k0 = 0; k0 < K; k0 += 16) {
        const uint64_t ad = desc(smem_u32(A) + (k0 >> 3) * 128, 128, sbo);
        const uint64_t bd = desc(smem_u32(B) + (k0 >> 3) * 128, 128, sbo);
        const uint32_t acc = (accumulate || k0 > 0) ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                     ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Bounded wait for the given phase; returns false (and sets *err) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase, int *err) {
    uint32_t done = 0;
    for (long long spins = 0; spins < (1ll << 26); ++spins) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_u32(mbar)), "r"(phase));
        if (done) return true;
    }
    if (err) atomicExch(err, 1);
    return false;
}

// 16 consecutive FP32 columns of this warp's 32 lanes (lane = row 32*warp + laneid)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(holder)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace tc
}  // namespace airga
