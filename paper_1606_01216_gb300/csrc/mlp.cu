// Learned SPAI-column predictor: a 16 -> 64 -> 64 -> 16 perceptron (ReLU,
// BF16 weights and activations, FP32 accumulation in tensor memory) that maps
// local features of column j of a shifted matrix A = s^2 M + s D + K (Eq. 1.1)
// to the seven entries of SPAI column j (Sec. 3.1, Eq. 3.1, pattern
// J_j = {j-3..j+3}), trained on the GPU on columns of exactly computed SPAIs.
// It stands in for the SPAI update of Sec. 3.2 when moving to a new shift.
//
// Features (FP32) of column j, n rows:
//   x = ( log10(s)/4, alpha, beta, log10(A_jj)/8,
//         A(j+d, j) / sqrt(A(j+d, j+d) A_jj) for d = -3,-2,-1,1,2,3 (0 outside),
//         min(j, 8)/8, min(n-1-j, 8)/8, j mod 2, 0, 0, 0 )
// Targets: t_o = P(j+d, j) sqrt(A(j+d, j+d) A_jj), d = o - 3, o = 0..6;
// output mask bit o set when 0 <= j+d < n.  Inference undoes the scaling.
//
// Kernels (all tensor-core work is tcgen05.mma, kind::f16, BF16 x BF16 -> FP32,
// M = 128 samples per tile, operands in shared memory in the no-swizzle
// K-major layout, accumulators in tensor memory):
//   mlp_features_kernel  one thread per column: features, targets, masks
//   mlp_infer_kernel     persistent, 128-sample tiles: 3 GEMMs; MODE 0 writes
//                        the outputs, MODE 1 computes the features from A's
//                        band and writes the decoded P band (learned SPAI)
//   mlp_train_kernel     persistent, 128-sample tiles: forward (3 GEMMs),
//                        backward (2 GEMMs for the hidden deltas, 2 GEMMs for
//                        all weight and bias gradients), gradients summed over
//                        the CTA's tiles in tensor memory, one partial per CTA
//   mlp_update_kernel    sums the CTA partials in a fixed order (FP64); either
//                        writes the mean gradient or takes an Adam step
//                        (Kingma and Ba, Algorithm 1) on the FP32 master
//                        parameters and refreshes their BF16 copies
// Weight gradients as GEMMs over the sample dimension: with K = 128 samples,
//   G2 = [dz2^T ; dY^T ; 0] (128 x 128) times [h1^T ; 1 ; 0]^T (80 x 128)
//        -> dW2 (rows 0..63, cols 0..63), db2 (rows 0..63, col 64),
//           db3 (rows 64..79, col 64)
//   G1 = [h2^T ; dz1^T] (128 x 128) times [dY^T ; x^T ; 1 ; 0]^T (48 x 128)
//        -> dW3^T (rows 0..63, cols 0..15), dW1 (rows 64..127, cols 16..31),
//           db1 (rows 64..127, col 32)
// so every gradient, biases included, comes out of two accumulating MMAs.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "airga_internal.cuh"
#include "ieee_conv.cuh"
#include "tc_common.cuh"

namespace airga {
namespace mlpdev {

constexpr int kIn = 16, kHid = 64, kOut = 16, kUsed = 7;
constexpr int kOffW1 = 0, kOffB1 = 1024, kOffW2 = 1088, kOffB2 = 5184, kOffW3 = 5248,
              kOffB3 = 6272, kNParam = 6288;
// BF16 weights in global memory, stored as the shared-memory operand image
// (K-major core-matrix layout) so a CTA stages them with straight 16-byte
// copies: W1 [64 x 16] | W2 [64 x 64] | W3 [16 x 64] (forward B operands) |
// W3^T [64 x 16] | W2^T [64 x 64] (backward B operands), bytes:
constexpr int kImgW1 = 0, kImgW2 = 2048, kImgW3 = 10240, kImgW3t = 12288, kImgW2t = 14336,
              kImgFwd = 12288, kImgAll = 22528;
constexpr int kTile = 128;
constexpr int kDistCap = 8;
constexpr long long kWaitNs = 2000000000ll;   // bound on any tensor-core completion wait
// error bits (OR-ed into a device int): bad sample index / column, non-positive
// or non-finite diagonal of A, tensor-core wait timeout.  Bit 0 is left to the
// SPAI rank flag that shares the preconditioner's status word.
constexpr int kFlagIndex = 8, kFlagDiag = 2, kFlagTimeout = 4;

using tc::kmaj_off;
using ieee::f64_to_f32;
using ieee::f32_to_f64;
using ieee::half_of;

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// 8 consecutive K elements (k0 % 8 == 0) of row r of a K-major operand
__device__ __forceinline__ void st8(uint8_t *base, int r, int k0, int K, const float *v) {
    uint4 q = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]),
                         pack2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(base + kmaj_off(r, k0, K)) = q;
}

__device__ __forceinline__ long long gtime() {
    long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for an MMA commit.  Thread 0 alone polls the mbarrier (the
// others wait at the CTA barrier and take no issue slots); the outcome is
// made uniform across the CTA.  On a timeout `code` is OR-ed into *err.
__device__ __forceinline__ bool wait_mma(uint64_t *mbar, uint32_t &phase, int *err, int code) {
    uint32_t done = 1;
    if (threadIdx.x == 0) {
        const uint32_t addr = tc::smem_u32(mbar);
        const long long t0 = gtime();
        // bounded by the timer and, should the timer stall, by a round count
        // (each round takes well over a nanosecond)
        for (long long round = 0; round < kWaitNs; ++round) {
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                         "selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(done)
                         : "r"(addr), "r"(phase));
            if (done || gtime() - t0 > kWaitNs) break;
        }
    }
    phase ^= 1u;
    const int ok = __syncthreads_and((int)done);
    tc::fence_after();
    if (!ok && threadIdx.x == 0 && err) atomicOr(err, code);
    return ok != 0;
}

// generic shared-memory writes and tensor-memory reads of all threads ->
// visible to / ordered before the next MMA issued by thread 0
__device__ __forceinline__ void sync_for_mma() {
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// 64 FP32 columns c0.. of this thread's tensor-memory lane, 16 at a time
template <int N>
__device__ __forceinline__ void tld(uint32_t taddr, float (&v)[N]) {
#pragma unroll
    for (int c = 0; c < N; c += 16) {
        float t[16];
        tc::tmem_ld16(taddr + c, t);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[c + k] = t[k];
    }
}

// ---------------------------------------------------------------------------
// features of column j (FP32 arithmetic: the network consumes BF16 operands,
// and FP64 square roots and divisions would dominate the learned build)
// ---------------------------------------------------------------------------
struct FeatConst {
    float f0, f1, f2;   // log10(s)/4, alpha, beta
};

__device__ __forceinline__ double band_at(const double *__restrict__ band, int64_t n, int64_t i, int d) {
    return band[(int64_t)(d + 3) * n + i];   // A(i, i+d)
}

// raw inputs of one row, fetched one tile ahead
struct RawRow {
    double dg[7];    // MODE 1: A(j+d, j+d), d = -3..3 (0 outside)
    double od[6];    // MODE 1: A(j+d, j), d = -3,-2,-1,1,2,3 (0 outside)
    float x[16];     // MODE 0: the feature row
};

// band values of column j of A (zeros when j is outside [0, n))
__device__ __forceinline__ void fetch_band_row(const double *__restrict__ A, int64_t n, int64_t j,
                                               RawRow &w) {
    const bool in = j >= 0 && j < n;
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        const int64_t i = j + o - 3;
        w.dg[o] = (in && i >= 0 && i < n) ? band_at(A, n, i, 0) : 0.0;
    }
    const int ds[6] = {-3, -2, -1, 1, 2, 3};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int64_t i = j + ds[c];
        w.od[c] = (in && i >= 0 && i < n) ? band_at(A, n, i, -ds[c]) : 0.0;
    }
}

// Features of column j from its band values (FP32 arithmetic: the network
// consumes BF16 operands, and FP64 square roots and divisions would dominate
// the learned build).  Returns false when a diagonal entry it needs is not
// positive and finite.  r[o] = 1 / sqrt(A(j+d, j+d)) for d = o - 3 (0 outside).
__device__ __forceinline__ bool row_features(const RawRow &w, int64_t n, int64_t j, const FeatConst &fc,
                                             float (&f)[16], float (&r)[7]) {
    bool ok = true;
    float dg[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) {
        const int64_t i = j + o - 3;
        r[o] = 0.0f;
        dg[o] = f64_to_f32(w.dg[o]);
        if (i >= 0 && i < n) {
            ok = ok && dg[o] > 0.0f && dg[o] < INFINITY;
            r[o] = rsqrtf(dg[o]);   // hardware reciprocal square root (<= 2 ulp)
        }
    }
    f[0] = fc.f0;
    f[1] = fc.f1;
    f[2] = fc.f2;
    f[3] = log10f(dg[3]) * 0.125f;
    const int ds[6] = {-3, -2, -1, 1, 2, 3};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const int64_t i = j + ds[c];
        f[4 + c] = (i >= 0 && i < n) ? (f64_to_f32(w.od[c]) * r[ds[c] + 3]) * r[3] : 0.0f;
    }
    const int d0 = j < kDistCap ? (int)j : kDistCap;
    const int d1 = n - 1 - j < kDistCap ? (int)(n - 1 - j) : kDistCap;
    f[10] = __int2float_rn(d0) * (1.0f / kDistCap);
    f[11] = __int2float_rn(d1) * (1.0f / kDistCap);
    f[12] = (j & 1) ? 1.0f : 0.0f;
    f[13] = f[14] = f[15] = 0.0f;
    return ok;
}

__global__ void mlp_features_kernel(const double *__restrict__ A, const double *__restrict__ P,
                                    int64_t n, const int64_t *__restrict__ cols, int64_t count,
                                    FeatConst fc, float *__restrict__ X, float *__restrict__ T,
                                    uint8_t *__restrict__ mask, int *__restrict__ err) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t j = cols ? cols[k] : k;
    if (j < 0 || j >= n) {
        atomicOr(err, kFlagIndex);
        return;
    }
    RawRow w;
    fetch_band_row(A, n, j, w);
    float f[16], rs[7];
    if (!row_features(w, n, j, fc, f, rs)) atomicOr(err, kFlagDiag);
    float4 *xr = reinterpret_cast<float4 *>(X + k * kIn);
#pragma unroll
    for (int q = 0; q < 4; ++q) xr[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
    if (!P) return;
    const double djj = band_at(A, n, j, 0);
    float t[8];
    unsigned m = 0;
#pragma unroll
    for (int o = 0; o < kUsed; ++o) {
        const int d = o - 3;
        const int64_t i = j + d;
        t[o] = 0.0f;
        if (i >= 0 && i < n) {
            t[o] = (float)(band_at(P, n, i, -d) * sqrt(band_at(A, n, i, 0) * djj));
            m |= 1u << o;
        }
    }
    t[7] = 0.0f;
    float4 *tr = reinterpret_cast<float4 *>(T + k * 8);
    tr[0] = make_float4(t[0], t[1], t[2], t[3]);
    tr[1] = make_float4(t[4], t[5], t[6], t[7]);
    mask[k] = (uint8_t)m;
}

// ---------------------------------------------------------------------------
// weight staging (once per CTA)
// ---------------------------------------------------------------------------
// copy BYTES of the weight image into shared memory with NT threads
template <int BYTES, int NT>
__device__ __forceinline__ void stage_image(const uint8_t *__restrict__ img, uint8_t *dst) {
    constexpr int kVec = BYTES / 16, kIt = (kVec + NT - 1) / NT;
    static_assert(kVec * 16 == BYTES, "image size");
    uint4 v[kIt];
    const uint4 *src = reinterpret_cast<const uint4 *>(img);
#pragma unroll
    for (int q = 0; q < kIt; ++q) {
        const int e = q * NT + (int)threadIdx.x;
        if (e < kVec) v[q] = src[e];
    }
#pragma unroll
    for (int q = 0; q < kIt; ++q) {
        const int e = q * NT + (int)threadIdx.x;
        if (e < kVec) reinterpret_cast<uint4 *>(dst)[e] = v[q];
    }
}

// write parameter k (a weight) into the image, at its forward position and,
// for W2 and W3, at its transposed position
__device__ __forceinline__ void image_put(uint8_t *img, int k, float w) {
    const __nv_bfloat16 b = __float2bfloat16(w);
    auto put = [&](int off) { *reinterpret_cast<__nv_bfloat16 *>(img + off) = b; };
    if (k < kOffB1) {
        const int o = k / kIn, i = k % kIn;
        put(kImgW1 + kmaj_off(o, i, kIn));
    } else if (k >= kOffW2 && k < kOffB2) {
        const int e = k - kOffW2, o = e / kHid, i = e % kHid;
        put(kImgW2 + kmaj_off(o, i, kHid));
        put(kImgW2t + kmaj_off(i, o, kHid));
    } else if (k >= kOffW3 && k < kOffB3) {
        const int e = k - kOffW3, o = e / kHid, h = e % kHid;
        put(kImgW3 + kmaj_off(o, h, kHid));
        put(kImgW3t + kmaj_off(h, o, kOut));
    }
}

// Thread roles inside a CTA of NT threads working on one 128-sample tile:
// warp w reads tensor-memory lanes 32 (w % 4) .. +31, i.e. sample rows
// r = 32 (w % 4) + lane, and takes column group q = w / 4 of QW = NT / 128
// groups (64 / QW columns of each hidden layer).

// ---------------------------------------------------------------------------
// inference
// ---------------------------------------------------------------------------
struct InferArgs {
    const uint8_t *wimg;
    const float *params;     // biases read from here
    int64_t count;           // samples (MODE 0) or columns n (MODE 1)
    const float *X;          // MODE 0: [count][16]
    float *Y;                // MODE 0: [count][16]
    const double *A;         // MODE 1: band of A
    double *P;               // MODE 1: band of the predicted P (written)
    double *Psym;            // MODE 1: band of 1/2 (P + P^T) (written)
    FeatConst fc;
    int *flag;               // MODE 1: status bits of the new preconditioner
};

// One warp group per CTA, several CTAs per SM: a tile's steps (features,
// three MMAs, two ReLU epilogues, output) form a dependent chain, and the
// chains of the CTAs sharing an SM overlap.  One 64-column tensor-memory
// accumulator serves all three layers and one shared-memory buffer both
// hidden layers (each is consumed before the next MMA overwrites it).
constexpr int kInferThreads = 128;
constexpr int kInferPerSm = 4;
constexpr int kInferSmem = kImgFwd + 4096 + 16384 + 4096 + 1024;   // image | X | H | P exchange | slack
constexpr uint32_t kInferCols = 64;
// MODE 1 tiles: 128 consecutive columns, of which the middle kOwn are owned;
// 3 halo columns on each side supply the transposed entries of P_sym.
constexpr int kHalo = 3, kOwn = kTile - 2 * kHalo;

template <int MODE>
__device__ __forceinline__ void fetch_row(const InferArgs &a, int64_t row, RawRow &w) {
    if (MODE == 0) {
        if (row < a.count) {
            const float4 *xr = reinterpret_cast<const float4 *>(a.X + row * kIn);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = xr[q];
                w.x[4 * q] = v.x;
                w.x[4 * q + 1] = v.y;
                w.x[4 * q + 2] = v.z;
                w.x[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) w.x[k] = 0.0f;
        }
    } else {
        fetch_band_row(a.A, a.count, row, w);
    }
}

template <int MODE>
__device__ __forceinline__ int64_t tile_row(int64_t tile, int r) {
    return MODE == 0 ? tile * kTile + r : tile * kOwn - kHalo + r;
}

template <int MODE>
__global__ void __launch_bounds__(kInferThreads, kInferPerSm) mlp_infer_kernel(InferArgs a) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sW1 = sm + kImgW1, *sW2 = sm + kImgW2, *sW3 = sm + kImgW3, *sX = sm + kImgFwd,
            *sH = sX + 4096;
    float(*sP)[8] = reinterpret_cast<float(*)[8]>(sH + 16384);   // MODE 1: P(j+d, j), d = o - 3
    __shared__ float sb[kHid + kHid + kOut];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r = tid;   // sample row = tensor-memory lane

    stage_image<kImgFwd, kInferThreads>(a.wimg, sm);
    for (int e = tid; e < kHid; e += blockDim.x) {
        sb[e] = a.params[kOffB1 + e];
        sb[kHid + e] = a.params[kOffB2 + e];
    }
    if (tid < kOut) sb[2 * kHid + tid] = a.params[kOffB3 + tid];
    if (warp == 0) tc::tmem_alloc(&tmem_holder, kInferCols);
    if (tid == 0) tc::mbar_init(&mbar);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool bad = false;

    const int64_t n = a.count;
    const int64_t ntiles = MODE == 0 ? (n + kTile - 1) / kTile : (n + kOwn - 1) / kOwn;
    RawRow nxt;
    int64_t tile = blockIdx.x;
    if (tile < ntiles) fetch_row<MODE>(a, tile_row<MODE>(tile, r), nxt);
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t row = tile_row<MODE>(tile, r);
        const bool valid = row >= 0 && row < n;
        float rs[7];
        {
            float f[16];
            if (MODE == 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k) f[k] = nxt.x[k];
            } else if (valid) {
                if (!row_features(nxt, n, row, a.fc, f, rs)) bad = true;
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) f[k] = 0.0f;
            }
            st8(sX, r, 0, kIn, f);
            st8(sX, r, 8, kIn, f + 8);
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem, sX, sW1, kIn, kHid, false);
            tc::commit(&mbar);
        }
        // fetch the next tile's inputs while this one runs
        if (tile + gridDim.x < ntiles) fetch_row<MODE>(a, tile_row<MODE>(tile + gridDim.x, r), nxt);
        if (!wait_mma(&mbar, phase, a.flag, kFlagTimeout)) break;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float z[16];
            tc::tmem_ld16(lane + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = fmaxf(z[k] + sb[c0 + k], 0.0f);
            st8(sH, r, c0, kHid, z);
            st8(sH, r, c0 + 8, kHid, z + 8);
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem, sH, sW2, kHid, kHid, false);
            tc::commit(&mbar);
        }
        if (!wait_mma(&mbar, phase, a.flag, kFlagTimeout)) break;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float z[16];
            tc::tmem_ld16(lane + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = fmaxf(z[k] + sb[kHid + c0 + k], 0.0f);
            st8(sH, r, c0, kHid, z);
            st8(sH, r, c0 + 8, kHid, z + 8);
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem, sH, sW3, kHid, kOut, false);
            tc::commit(&mbar);
        }
        if (!wait_mma(&mbar, phase, a.flag, kFlagTimeout)) break;
        float y[16];
        tc::tmem_ld16(lane, y);
#pragma unroll
        for (int o = 0; o < 16; ++o) y[o] += sb[2 * kHid + o];
        if (MODE == 0) {
            if (valid) {
                float4 *yr = reinterpret_cast<float4 *>(a.Y + row * kOut);
#pragma unroll
                for (int v = 0; v < 4; ++v) yr[v] = make_float4(y[4 * v], y[4 * v + 1], y[4 * v + 2], y[4 * v + 3]);
            }
        } else {
            // P(j+d, j) = y_o / sqrt(A(j+d, j+d) A_jj), exchanged through shared memory
#pragma unroll
            for (int o = 0; o < kUsed; ++o) sP[r][o] = valid ? (y[o] * rs[o]) * rs[3] : 0.0f;
            __syncthreads();
            const bool owned = r >= kHalo && r < kTile - kHalo && valid;
            if (owned) {
                const int64_t i = row;   // this thread writes row i of P and of P_sym
#pragma unroll
                for (int dp = -3; dp <= 3; ++dp) {
                    const int64_t c = i + dp;
                    double p = 0.0, ps = 0.0;
                    if (c >= 0 && c < n) {
                        const float pic = sP[r + dp][3 - dp];   // P(i, c): column c, offset -dp
                        const float pci = sP[r][3 + dp];        // P(c, i): column i, offset +dp
                        p = f32_to_f64(pic);
                        ps = half_of(p + f32_to_f64(pci));
                    }
                    a.P[(int64_t)(dp + 3) * n + i] = p;
                    a.Psym[(int64_t)(dp + 3) * n + i] = ps;
                }
            }
        }
        tc::fence_before();   // tensor-memory reads (and the P exchange) done before the next tile
        __syncthreads();
        tc::fence_after();
    }
    if (MODE == 1 && bad) atomicOr(a.flag, kFlagDiag);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_free(tmem, kInferCols);
}

// ---------------------------------------------------------------------------
// training: forward + backward, per-CTA gradient partials
// ---------------------------------------------------------------------------
struct TrainArgs {
    const uint8_t *wimg;
    const float *params;
    const float *X;          // [N][16]
    const float *T;          // [N][8]
    const uint8_t *mask;     // [N]
    int64_t N;
    const int32_t *idx;      // [B] sample indices, or null: counter-based draw
    int32_t B;
    uint64_t seed;
    int64_t *step;           // step[0] completed steps (read), step[1] <- step[0] + 1; null = no counter
    float *gpart;            // [grid][kNParam]
    double *lpart;           // [grid] sum of squared masked errors
    int *err;
};

constexpr int kTrainThreads = 512;   // four column groups of 16 columns
// smem offsets (bytes from the 1024-aligned base); the first kImgAll bytes
// mirror the weight image
constexpr int kTsW1 = kImgW1, kTsW2 = kImgW2, kTsW3 = kImgW3, kTsW3t = kImgW3t, kTsW2t = kImgW2t,
              kTsX = kImgAll, kTsH1 = kTsX + 4096, kTsH2 = kTsH1 + 16384, kTsDY = kTsH2 + 16384,
              kTsDZ2 = kTsDY + 4096, kTsTA1 = kTsDZ2 + 16384, kTsTA2 = kTsTA1 + 32768,
              kTsB2 = kTsTA2 + 32768, kTsB1 = kTsB2 + 20480, kTsEnd = kTsB1 + 12288;
constexpr int kTrainSmem = kTsEnd + 1024;
constexpr uint32_t kTrainCols = 512;
// tensor-memory columns
constexpr uint32_t kCZ1 = 0, kCZ2 = 64, kCY = 128, kCDH2 = 160, kCDH1 = 224, kCG2 = 288, kCG1 = 384;

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) applied to
// the counter seed + (c + 1) * golden gamma: output number c of the sequence.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// 4 consecutive K elements (k0 % 4 == 0) of row r of a K-major operand
__device__ __forceinline__ void st4(uint8_t *base, int r, int k0, int K, const float *v) {
    *reinterpret_cast<uint2 *>(base + kmaj_off(r, k0, K)) = make_uint2(pack2(v[0], v[1]), pack2(v[2], v[3]));
}

__global__ void __launch_bounds__(kTrainThreads, 1) mlp_train_kernel(TrainArgs a) {
    constexpr int NT = kTrainThreads;
    extern __shared__ uint8_t smraw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sW1 = sm + kTsW1, *sW2 = sm + kTsW2, *sW3 = sm + kTsW3, *sW3t = sm + kTsW3t,
            *sW2t = sm + kTsW2t, *sX = sm + kTsX, *sH1 = sm + kTsH1, *sH2 = sm + kTsH2,
            *sDY = sm + kTsDY, *sDZ2 = sm + kTsDZ2, *TA1 = sm + kTsTA1, *TA2 = sm + kTsTA2,
            *B2 = sm + kTsB2, *B1 = sm + kTsB1;
    __shared__ float sb[kHid + kHid + kOut];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    __shared__ double sred[NT / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane_id = tid & 31;
    const int rg = warp & 3, q = warp >> 2;     // lane group, column group (16 hidden columns)
    const int r = rg * 32 + lane_id;            // sample row of this thread
    const int c0 = q * 16;
    constexpr int KS = kTile;   // K of the weight-gradient GEMMs (samples)

    int64_t step0 = 0;
    if (a.step) {
        step0 = a.step[0];
        if (blockIdx.x == 0 && tid == 0) a.step[1] = step0 + 1;
    }

    // weights, transposed weights, constant rows
    stage_image<kImgAll, NT>(a.wimg, sm);
    const __nv_bfloat16 one = __float2bfloat16(1.0f), zero = __float2bfloat16(0.0f);
    for (int e = tid; e < 16 * KS; e += NT) {
        const int rr = e / KS, cc = e % KS;
        *reinterpret_cast<__nv_bfloat16 *>(B2 + kmaj_off(64 + rr, cc, KS)) = rr == 0 ? one : zero;
        *reinterpret_cast<__nv_bfloat16 *>(B1 + kmaj_off(32 + rr, cc, KS)) = rr == 0 ? one : zero;
    }
    for (int e = tid; e < 48 * KS; e += NT) {
        const int rr = e / KS, cc = e % KS;
        *reinterpret_cast<__nv_bfloat16 *>(TA2 + kmaj_off(80 + rr, cc, KS)) = zero;
    }
    for (int e = tid; e < kHid; e += NT) {
        sb[e] = a.params[kOffB1 + e];
        sb[kHid + e] = a.params[kOffB2 + e];
    }
    if (tid < kOut) sb[2 * kHid + tid] = a.params[kOffB3 + tid];
    if (warp == 0) tc::tmem_alloc(&tmem_holder, kTrainCols);
    if (tid == 0) tc::mbar_init(&mbar);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_holder;
    const uint32_t lane = tmem + ((uint32_t)(rg * 32) << 16);
    uint32_t phase = 0;
    float lsum = 0.0f;   // this thread's squared errors (a few tiles at most per launch)
    bool alive = true;

    const int64_t ntiles = ((int64_t)a.B + kTile - 1) / kTile;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x, ++it) {
        // ---- samples of this tile: group q loads features 4q..4q+3 and, for q < 2,
        //      targets 4q..4q+3 and the mask ----
        const int64_t b = tile * kTile + r;
        int64_t si = -1;
        if (b < a.B) {
            if (a.idx) {
                si = a.idx[b];
                if (si < 0 || si >= a.N) {
                    if (q == 0) atomicOr(a.err, kFlagIndex);
                    si = -1;
                }
            } else {
                si = (int64_t)(splitmix64(a.seed, (uint64_t)step0 * 0x100000000ull + (uint64_t)b) %
                               (uint64_t)a.N);
            }
        }
        float f[4] = {0.0f, 0.0f, 0.0f, 0.0f}, tg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        unsigned mk = 0;
        if (si >= 0) {
            const float4 v = reinterpret_cast<const float4 *>(a.X + si * kIn)[q];
            f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
            if (q < 2) {
                const float4 t = reinterpret_cast<const float4 *>(a.T + si * 8)[q];
                tg[0] = t.x; tg[1] = t.y; tg[2] = t.z; tg[3] = t.w;
                mk = a.mask[si];
            }
        }
        st4(sX, r, 4 * q, kIn, f);
#pragma unroll
        for (int k = 0; k < 4; ++k) tc::st_bf16(B1, 16 + 4 * q + k, r, KS, f[k]);   // x^T
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCZ1, sX, sW1, kIn, kHid, false);
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;

        // ---- h1 (columns c0..c0+15) ----
        {
            float z[16];
            tc::tmem_ld16(lane + kCZ1 + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = fmaxf(z[k] + sb[c0 + k], 0.0f);
            st8(sH1, r, c0, kHid, z);
            st8(sH1, r, c0 + 8, kHid, z + 8);
#pragma unroll
            for (int k = 0; k < 16; ++k) tc::st_bf16(B2, c0 + k, r, KS, z[k]);   // h1^T
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCZ2, sH1, sW2, kHid, kHid, false);
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;

        // ---- h2 ----
        {
            float z[16];
            tc::tmem_ld16(lane + kCZ2 + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = fmaxf(z[k] + sb[kHid + c0 + k], 0.0f);
            st8(sH2, r, c0, kHid, z);
            st8(sH2, r, c0 + 8, kHid, z + 8);
#pragma unroll
            for (int k = 0; k < 16; ++k) tc::st_bf16(TA1, c0 + k, r, KS, z[k]);   // h2^T
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCY, sH2, sW3, kHid, kOut, false);
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;

        // ---- output error e = mask (y - t), outputs 4q..4q+3 ----
        {
            float y[16];
            tc::tmem_ld16(lane + kCY, y);
            float e[4];
            float l = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = 4 * q + k;
                const float yo = q == 0 ? y[k] : (q == 1 ? y[4 + k] : (q == 2 ? y[8 + k] : y[12 + k]));
                e[k] = (o < kUsed && ((mk >> o) & 1u)) ? (yo + sb[2 * kHid + o]) - tg[k] : 0.0f;
                l += e[k] * e[k];
            }
            lsum += l;
            st4(sDY, r, 4 * q, kOut, e);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                tc::st_bf16(B1, 4 * q + k, r, KS, e[k]);        // dY^T (B operand of G1)
                tc::st_bf16(TA2, 64 + 4 * q + k, r, KS, e[k]);  // dY^T (A rows of G2)
            }
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCDH2, sDY, sW3t, kOut, kHid, false);   // dh2 = dY W3
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;

        // ---- dz2 = dh2 relu'(z2) ----
        {
            float g[16], z[16];
            tc::tmem_ld16(lane + kCDH2 + c0, g);
            tc::tmem_ld16(lane + kCZ2 + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = (z[k] + sb[kHid + c0 + k] > 0.0f) ? g[k] : 0.0f;
            st8(sDZ2, r, c0, kHid, g);
            st8(sDZ2, r, c0 + 8, kHid, g + 8);
#pragma unroll
            for (int k = 0; k < 16; ++k) tc::st_bf16(TA2, c0 + k, r, KS, g[k]);   // dz2^T
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCDH1, sDZ2, sW2t, kHid, kHid, false);   // dh1 = dz2 W2
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;

        // ---- dz1 = dh1 relu'(z1) ----
        {
            float g[16], z[16];
            tc::tmem_ld16(lane + kCDH1 + c0, g);
            tc::tmem_ld16(lane + kCZ1 + c0, z);
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = (z[k] + sb[c0 + k] > 0.0f) ? g[k] : 0.0f;
#pragma unroll
            for (int k = 0; k < 16; ++k) tc::st_bf16(TA1, 64 + c0 + k, r, KS, g[k]);   // dz1^T
        }
        sync_for_mma();
        if (tid == 0) {
            tc::gemm(tmem + kCG2, TA2, B2, KS, 80, it > 0);
            tc::gemm(tmem + kCG1, TA1, B1, KS, 48, it > 0);
            tc::commit(&mbar);
        }
        if (!(alive = wait_mma(&mbar, phase, a.err, kFlagTimeout))) break;
        tc::fence_before();
    }

    // ---- per-CTA partials out of tensor memory (column group q takes one
    //      16-column slice of G2 cols 0..63, plus one of the remaining slices) ----
    float *gp = a.gpart + (size_t)blockIdx.x * kNParam;
    if (alive && it > 0) {
        {
            float v[16];
            tc::tmem_ld16(lane + kCG2 + c0, v);    // dW2 rows 0..63, columns c0..c0+15
            if (r < 64)
#pragma unroll
                for (int k = 0; k < 16; ++k) gp[kOffW2 + r * kHid + c0 + k] = v[k];
        }
        float v[16];
        if (q == 0) {
            tc::tmem_ld16(lane + kCG2 + 64, v);    // col 64: db2 (rows < 64), db3 (rows 64..79)
            if (r < 64) gp[kOffB2 + r] = v[0];
            else if (r < 80) gp[kOffB3 + r - 64] = v[0];
        } else if (q == 1) {
            tc::tmem_ld16(lane + kCG1, v);          // cols 0..15: dW3^T rows 0..63
            if (r < 64)
#pragma unroll
                for (int o = 0; o < 16; ++o) gp[kOffW3 + o * kHid + r] = v[o];
        } else if (q == 2) {
            tc::tmem_ld16(lane + kCG1 + 16, v);     // cols 16..31: dW1 rows 64..127
            if (r >= 64)
#pragma unroll
                for (int k = 0; k < 16; ++k) gp[kOffW1 + (r - 64) * kIn + k] = v[k];
        } else {
            tc::tmem_ld16(lane + kCG1 + 32, v);     // col 32: db1 rows 64..127
            if (r >= 64) gp[kOffB1 + r - 64] = v[0];
        }
    } else {
        for (int k = tid; k < kNParam; k += NT) gp[k] = 0.0f;
    }
    // loss partial (fixed-order reduction)
    double l = (double)lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if (lane_id == 0) sred[warp] = l;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sred[w];
        a.lpart[blockIdx.x] = t;
    }
    if (warp == 0) tc::tmem_free(tmem, kTrainCols);
}

// ---------------------------------------------------------------------------
// partial sums -> mean gradient, or Adam step
// ---------------------------------------------------------------------------
struct UpdateArgs {
    float *params, *m, *v;
    uint8_t *wimg;
    const float *gpart;
    const double *lpart;
    int G;
    int32_t B;
    float *grad_out;     // mode 0
    double *loss_d;      // mode 0 (double loss) or null
    float *loss_f;       // mode 1 (loss of this step) or null
    float lr, beta1, beta2, eps;
    int32_t cosine_steps;
    int64_t *step;       // mode 1: t = step[1]; step[0] <- t
    int mode;            // 0 gradient, 1 Adam
};

// Block of 256 threads = 32 parameters x 8 slices of the CTA partials; each
// slice sums its partials in CTA order, then the 8 slice sums are added in
// slice order (a fixed order: results are reproducible run to run).
constexpr int kUpdParams = 32, kUpdSlices = 8;

__global__ void __launch_bounds__(kUpdParams * kUpdSlices) mlp_update_kernel(UpdateArgs a) {
    __shared__ double red[kUpdSlices][kUpdParams];
    const int lane = threadIdx.x % kUpdParams, sl = threadIdx.x / kUpdParams;
    const int k = blockIdx.x * kUpdParams + lane;
    const double invB = 1.0 / (double)a.B;
    double g = 0.0;
    if (k < kNParam) {
#pragma unroll 4
        for (int c = sl; c < a.G; c += kUpdSlices) g += (double)a.gpart[(size_t)c * kNParam + k];
    }
    red[sl][lane] = g;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double l = 0.0;
        for (int c = 0; c < a.G; ++c) l += a.lpart[c];
        l *= 0.5 * invB;
        if (a.loss_d) *a.loss_d = l;
        if (a.loss_f) *a.loss_f = (float)l;
    }
    __syncthreads();
    if (sl != 0 || k >= kNParam) return;
    g = 0.0;
#pragma unroll
    for (int t = 0; t < kUpdSlices; ++t) g += red[t][lane];
    g *= invB;
    if (a.mode == 0) {
        a.grad_out[k] = (float)g;
        return;
    }
    const int64_t t = a.step[1];
    double lr = a.lr;
    if (a.cosine_steps > 0) {
        const double tt = (double)(t < a.cosine_steps ? t : a.cosine_steps);
        lr = a.lr * 0.5 * (1.0 + cos(3.14159265358979323846 * tt / (double)a.cosine_steps));
    }
    const double b1 = a.beta1, b2 = a.beta2;
    const double m = b1 * (double)a.m[k] + (1.0 - b1) * g;
    const double v = b2 * (double)a.v[k] + (1.0 - b2) * g * g;
    const double mhat = m / (1.0 - pow(b1, (double)t));
    const double vhat = v / (1.0 - pow(b2, (double)t));
    const float p = (float)((double)a.params[k] - lr * mhat / (sqrt(vhat) + (double)a.eps));
    a.m[k] = (float)m;
    a.v[k] = (float)v;
    a.params[k] = p;
    image_put(a.wimg, k, p);
    if (k == 0) a.step[0] = t;
}

__global__ void mlp_image_kernel(const float *__restrict__ params, uint8_t *__restrict__ img) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kNParam) image_put(img, k, params[k]);
}

}  // namespace mlpdev
}  // namespace airga

// ---------------------------------------------------------------------------
// handle and C ABI
// ---------------------------------------------------------------------------
using namespace airga;
using namespace airga::mlpdev;

struct airga_mlp_s {
    std::shared_ptr<void> mem;    // params | m | v (FP32) | BF16 weight image | step[2] | err
    float *params = nullptr, *m = nullptr, *v = nullptr;
    uint8_t *wimg = nullptr;        // BF16 weight image (kImgAll bytes)
    int64_t *step = nullptr;
    int *err = nullptr;
    std::shared_ptr<void> scratch;   // gpart [G][NP] floats | lpart [G] doubles
    float *gpart = nullptr;
    double *lpart = nullptr;
    int gmax = 0;
    int device = 0;
};

namespace {

int mlp_prepare(int dev_sms_dummy = 0) {
    (void)dev_sms_dummy;
    static thread_local int done_dev = -1;
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    if (done_dev == dev) return AIRGA_OK;
    AIRGA_CUDA(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmem));
    AIRGA_CUDA(cudaFuncSetAttribute(mlp_infer_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem));
    AIRGA_CUDA(cudaFuncSetAttribute(mlp_infer_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInferSmem));
    done_dev = dev;
    return AIRGA_OK;
}

int sm_count(int *out) {
    int dev = 0;
    AIRGA_CUDA(cudaGetDevice(&dev));
    AIRGA_CUDA(cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev));
    return AIRGA_OK;
}

// host SplitMix64 stream for the initial weights
struct SplitMix {
    uint64_t x;
    uint64_t next() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

int check_net(airga_mlp net) {
    if (!net || !net->params) return fail(AIRGA_E_INVALID_ARG, "network handle is NULL");
    return AIRGA_OK;
}

int launch_infer(int mode, const InferArgs &a, cudaStream_t s) {
    int st = mlp_prepare();
    if (st) return st;
    int sms = 0;
    st = sm_count(&sms);
    if (st) return st;
    const int64_t ntiles = mode == 0 ? (a.count + kTile - 1) / kTile : (a.count + kOwn - 1) / kOwn;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)kInferPerSm * sms);
    if (grid < 1) return AIRGA_OK;
    if (mode == 0) mlp_infer_kernel<0><<<grid, kInferThreads, kInferSmem, s>>>(a);
    else mlp_infer_kernel<1><<<grid, kInferThreads, kInferSmem, s>>>(a);
    AIRGA_CUDA(cudaGetLastError());
    return AIRGA_OK;
}

int launch_train(airga_mlp net, const float *X, const float *T, const uint8_t *mask, int64_t N,
                 const int32_t *idx, int32_t B, uint64_t seed, bool count_step, cudaStream_t s,
                 int *grid_out) {
    int st = mlp_prepare();
    if (st) return st;
    const int64_t ntiles = ((int64_t)B + kTile - 1) / kTile;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)net->gmax);
    TrainArgs a;
    a.wimg = net->wimg;
    a.params = net->params;
    a.X = X;
    a.T = T;
    a.mask = mask;
    a.N = N;
    a.idx = idx;
    a.B = B;
    a.seed = seed;
    a.step = count_step ? net->step : nullptr;
    a.gpart = net->gpart;
    a.lpart = net->lpart;
    a.err = net->err;
    mlp_train_kernel<<<grid, kTrainThreads, kTrainSmem, s>>>(a);
    AIRGA_CUDA(cudaGetLastError());
    *grid_out = grid;
    return AIRGA_OK;
}

}  // namespace

extern "C" {

void airga_mlp_train_options_default(airga_mlp_train_options *o) {
    if (!o) return;
    o->lr = 2e-3f;
    o->beta1 = 0.9f;
    o->beta2 = 0.999f;
    o->eps = 1e-8f;
    o->batch = 4096;
    o->cosine_steps = 0;
    o->seed = 0x5eed5eedull;
}

int airga_mlp_create(uint64_t seed, void *stream, airga_mlp *out) {
    if (!out) return fail(AIRGA_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    int st = sm_count(&sms);
    if (st) return st;
    auto *net = new airga_mlp_s;
    cudaGetDevice(&net->device);
    const size_t b_par = 256 * ((3 * sizeof(float) * kNParam + 255) / 256);
    const size_t b_wb = 256 * (((size_t)kImgAll + 255) / 256);
    st = make_buf(b_par + b_wb + 256, s, &net->mem);
    if (!st) st = make_buf(sizeof(float) * (size_t)kNParam * sms + sizeof(double) * sms, s, &net->scratch);
    if (st) {
        delete net;
        return st;
    }
    char *base = (char *)net->mem.get();
    net->params = (float *)base;
    net->m = net->params + kNParam;
    net->v = net->m + kNParam;
    net->wimg = (uint8_t *)(base + b_par);
    net->step = (int64_t *)(base + b_par + b_wb);
    net->err = (int *)(net->step + 2);
    net->gpart = (float *)net->scratch.get();
    net->lpart = (double *)(net->gpart + (size_t)kNParam * sms);
    net->gmax = sms;
    // Glorot-uniform weights, zero biases
    std::vector<float> h(kNParam, 0.0f);
    SplitMix rng{seed};
    struct L { int off, o, i; } layers[3] = {{kOffW1, kHid, kIn}, {kOffW2, kHid, kHid}, {kOffW3, kOut, kHid}};
    for (const L &l : layers) {
        const double lim = std::sqrt(6.0 / (double)(l.o + l.i));
        for (int e = 0; e < l.o * l.i; ++e) h[l.off + e] = (float)((2.0 * rng.uniform() - 1.0) * lim);
    }
    cudaError_t e = cudaMemcpyAsync(net->params, h.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->m, 0, sizeof(float) * 2 * kNParam, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->step, 0, 2 * sizeof(int64_t) + sizeof(int), s);
    if (e == cudaSuccess) {
        mlp_image_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(net->params, net->wimg);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vector goes out of scope
    if (e != cudaSuccess) {
        delete net;
        return cuda_fail(e, "mlp create");
    }
    *out = net;
    return AIRGA_OK;
}

int airga_mlp_set_params(airga_mlp net, const float *params, void *stream) {
    int st = check_net(net);
    if (st) return st;
    if (!params) return fail(AIRGA_E_INVALID_ARG, "params is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    AIRGA_CUDA(cudaMemcpyAsync(net->params, params, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, s));
    AIRGA_CUDA(cudaMemsetAsync(net->m, 0, sizeof(float) * 2 * kNParam, s));
    AIRGA_CUDA(cudaMemsetAsync(net->step, 0, 2 * sizeof(int64_t) + sizeof(int), s));
    mlp_image_kernel<<<(kNParam + 255) / 256, 256, 0, s>>>(net->params, net->wimg);
    AIRGA_CUDA(cudaGetLastError());
    return AIRGA_OK;
}

int airga_mlp_get_params(airga_mlp net, float *params, void *stream) {
    int st = check_net(net);
    if (st) return st;
    if (!params) return fail(AIRGA_E_INVALID_ARG, "params is NULL");
    AIRGA_CUDA(cudaMemcpyAsync(params, net->params, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
    return AIRGA_OK;
}

int airga_mlp_status(airga_mlp net, int64_t *steps_done, int *status_out, void *stream) {
    int st = check_net(net);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t h[2] = {0, 0};
    int herr = 0;
    AIRGA_CUDA(cudaMemcpyAsync(h, net->step, sizeof(h), cudaMemcpyDeviceToHost, s));
    AIRGA_CUDA(cudaMemcpyAsync(&herr, net->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AIRGA_CUDA(cudaStreamSynchronize(s));
    if (steps_done) *steps_done = h[0];
    if (status_out)
        *status_out = herr == 0 ? AIRGA_OK : ((herr & kFlagTimeout) ? AIRGA_E_TIMEOUT : AIRGA_E_INVALID_ARG);
    return AIRGA_OK;
}

int airga_mlp_features(airga_mat A, airga_precond P, double s, double alpha, double beta,
                       const int64_t *cols, int64_t count, float *X, float *T, uint8_t *mask,
                       int32_t *flag, void *stream) {
    int st = check_mat(A, "A");
    if (st) return st;
    if (!(s > 0.0) || !std::isfinite(s)) return fail(AIRGA_E_INVALID_ARG, "shift s must be positive and finite");
    if (count < 0 || (count > 0 && !X) || !flag) return fail(AIRGA_E_INVALID_ARG, "bad feature buffers");
    if (!cols && count > A->n) return fail(AIRGA_E_SHAPE, "count exceeds the rows of A without a column list");
    if (P && (P->n != A->n || P->factors.size() != 1))
        return fail(AIRGA_E_INVALID_ARG, "P must be a single factor of A's size");
    if (P && (!T || !mask)) return fail(AIRGA_E_INVALID_ARG, "T and mask are required with P");
    if (((uintptr_t)X & 15u) || (T && ((uintptr_t)T & 15u)))
        return fail(AIRGA_E_INVALID_ARG, "X and T must be 16-byte aligned");
    if (count == 0) return AIRGA_OK;
    FeatConst fc{(float)(std::log10(s) / 4.0), (float)alpha, (float)beta};
    const int threads = 256;
    const int64_t blocks = (count + threads - 1) / threads;
    mlp_features_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        A->band->d, P ? P->factors[0]->d : nullptr, A->n, cols, count, fc, X, P ? T : nullptr,
        P ? mask : nullptr, flag);
    AIRGA_CUDA(cudaGetLastError());
    return AIRGA_OK;
}

int airga_mlp_forward(airga_mlp net, const float *X, int64_t count, float *Y, void *stream) {
    TraceScope trace_("airga_mlp_forward", stream);
    int st = check_net(net);
    if (st) return st;
    if (count < 0 || (count > 0 && (!X || !Y))) return fail(AIRGA_E_INVALID_ARG, "bad forward buffers");
    if (((uintptr_t)X & 15u) || ((uintptr_t)Y & 15u))
        return fail(AIRGA_E_INVALID_ARG, "X and Y must be 16-byte aligned");
    if (count == 0) return AIRGA_OK;
    InferArgs a{};
    a.wimg = net->wimg;
    a.params = net->params;
    a.count = count;
    a.X = X;
    a.Y = Y;
    a.flag = net->err;
    return launch_infer(0, a, (cudaStream_t)stream);
}

int airga_mlp_grad(airga_mlp net, const float *X, const float *T, const uint8_t *mask, int64_t count,
                   const int32_t *idx, int32_t batch, float *grad, double *loss, void *stream) {
    int st = check_net(net);
    if (st) return st;
    if (count < 1 || count > INT32_MAX || batch < 1 || !X || !T || !mask || !idx || !grad)
        return fail(AIRGA_E_INVALID_ARG, "bad gradient arguments");
    if (((uintptr_t)X & 15u) || ((uintptr_t)T & 15u))
        return fail(AIRGA_E_INVALID_ARG, "X and T must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int grid = 0;
    st = launch_train(net, X, T, mask, count, idx, batch, 0, false, s, &grid);
    if (st) return st;
    UpdateArgs u{};
    u.gpart = net->gpart;
    u.lpart = net->lpart;
    u.G = grid;
    u.B = batch;
    u.grad_out = grad;
    u.loss_d = loss;
    u.mode = 0;
    mlp_update_kernel<<<(kNParam + kUpdParams - 1) / kUpdParams, kUpdParams * kUpdSlices, 0, s>>>(u);
    AIRGA_CUDA(cudaGetLastError());
    return AIRGA_OK;
}

int airga_mlp_train(airga_mlp net, const float *X, const float *T, const uint8_t *mask, int64_t count,
                    int32_t steps, const airga_mlp_train_options *opt, const int32_t *idx,
                    float *loss_hist, void *stream) {
    TraceScope trace_("airga_mlp_train", stream);
    int st = check_net(net);
    if (st) return st;
    airga_mlp_train_options o;
    airga_mlp_train_options_default(&o);
    if (opt) o = *opt;
    if (count < 1 || steps < 0 || o.batch < 1 || !X || !T || !mask || !(o.lr >= 0.0f) ||
        !(o.beta1 >= 0.0f && o.beta1 < 1.0f) || !(o.beta2 >= 0.0f && o.beta2 < 1.0f) || !(o.eps > 0.0f))
        return fail(AIRGA_E_INVALID_ARG, "bad training arguments");
    if (idx && count > INT32_MAX) return fail(AIRGA_E_INVALID_ARG, "explicit indices need count < 2^31");
    if (((uintptr_t)X & 15u) || ((uintptr_t)T & 15u))
        return fail(AIRGA_E_INVALID_ARG, "X and T must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t k = 0; k < steps; ++k) {
        int grid = 0;
        st = launch_train(net, X, T, mask, count, idx ? idx + (size_t)k * o.batch : nullptr, o.batch,
                          o.seed, true, s, &grid);
        if (st) return st;
        UpdateArgs u{};
        u.params = net->params;
        u.m = net->m;
        u.v = net->v;
        u.wimg = net->wimg;
        u.gpart = net->gpart;
        u.lpart = net->lpart;
        u.G = grid;
        u.B = o.batch;
        u.loss_f = loss_hist ? loss_hist + k : nullptr;
        u.lr = o.lr;
        u.beta1 = o.beta1;
        u.beta2 = o.beta2;
        u.eps = o.eps;
        u.cosine_steps = o.cosine_steps;
        u.step = net->step;
        u.mode = 1;
        mlp_update_kernel<<<(kNParam + kUpdParams - 1) / kUpdParams, kUpdParams * kUpdSlices, 0, s>>>(u);
        AIRGA_CUDA(cudaGetLastError());
    }
    return AIRGA_OK;
}

int airga_mlp_spai(airga_mlp net, airga_mat A, double s, double alpha, double beta, void *stream,
                   airga_precond *P_out) {
    TraceScope trace_("airga_mlp_spai", stream);
    if (!P_out) return fail(AIRGA_E_INVALID_ARG, "P_out is NULL");
    *P_out = nullptr;
    int st = check_net(net);
    if (!st) st = check_mat(A, "A");
    if (st) return st;
    if (!(s > 0.0) || !std::isfinite(s)) return fail(AIRGA_E_INVALID_ARG, "shift s must be positive and finite");
    cudaStream_t cs = (cudaStream_t)stream;
    auto *P = new airga_precond_s;
    P->n = A->n;
    BandPtr F;
    st = make_band(A->n, cs, &F);
    if (!st) st = make_band(A->n, cs, &P->psym);
    if (!st) st = make_buf(sizeof(int32_t), cs, &P->rank_flag);
    if (!st) {
        cudaError_t e = cudaMemsetAsync(P->rank_flag.get(), 0, sizeof(int32_t), cs);
        if (e != cudaSuccess) st = cuda_fail(e, "memset");
    }
    if (!st) {
        InferArgs a{};
        a.wimg = net->wimg;
        a.params = net->params;
        a.count = A->n;
        a.A = A->band->d;
        a.P = F->d;
        a.Psym = P->psym->d;
        a.fc = FeatConst{(float)(std::log10(s) / 4.0), (float)alpha, (float)beta};
        a.flag = (int *)P->rank_flag.get();
        st = launch_infer(1, a, cs);
    }
    if (st) {
        delete P;
        return st;
    }
    P->factors.push_back(F);
    *P_out = P;
    return AIRGA_OK;
}

void airga_mlp_free(airga_mlp net) { delete net; }

}  // extern "C"
