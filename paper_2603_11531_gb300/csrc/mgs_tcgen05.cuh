// Eq. 4 MLP on the 5th-generation tensor cores (tcgen05, sm_100-family):
// one CTA of 256 threads evaluates 256 Gaussians per step as two M = 128
// tiles that share one copy of the weights.
//
//   operands   shared memory, canonical no-swizzle K-major layout: 8-row x
//              16-byte core matrices stored contiguously (128 B each), core
//              matrices adjacent in K 128 B apart (leading byte offset),
//              adjacent in M/N (K/8) x 128 B apart (stride byte offset);
//   issue      one thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//              accumulate) for each K = 16 step and commits to an mbarrier;
//   result     accumulators live in TMEM (128 columns per CTA: tile 0 in
//              columns 0-63, tile 1 in 64-127, layer 2 reusing layer 1's
//              columns once they are read); thread t reads row t % 128 of tile
//              t / 128 with tcgen05.ld.32x32b (warp w sees lanes 32 (w % 4)..);
//   head       the 64 -> 5 head (BF16 h2, FP32 accumulate) runs on the CUDA
//              cores from the thread's own row, saving a third round trip.
//
// Every wait on the mbarrier is bounded; on timeout the kernel records an
// error flag in the workspace status and carries on (the host reports
// MGS_ERR_TIMEOUT at the next sync).
#pragma once

#include "mgs_internal.cuh"

namespace mgs {
static_assert(kMlpOut == 5, "the CUDA-core heads below unroll five outputs");
namespace tc {

constexpr int kRows = 128;          // rows per MMA tile
constexpr int kTiles = 2;           // tiles per CTA step
constexpr int kThreads = kRows * kTiles;
constexpr int kTmemCols = 128;
constexpr unsigned kWaitLimit = 1u << 22;

// byte offset of element (row, k) in a K-major canonical tile with K columns
__device__ __forceinline__ uint32_t core_off(int row, int k, int K) {
    return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     mbar)
                 : "memory");
}

// Bounded wait for the mbarrier phase; returns false on timeout.
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t phase) {
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane, without waiting.
__device__ __forceinline__ void ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory of the tcgen05 MLP (operands in canonical layout).
struct Smem {
    alignas(128) __nv_bfloat16 x[kTiles][kRows * kMlpK1];       // A of layer 1, K = 32
    alignas(128) __nv_bfloat16 h1[kTiles][kRows * kMlpHidden];  // A of layer 2, K = 64
    alignas(128) __nv_bfloat16 w1[kMlpHidden * kMlpK1];         // B, N = 64, K = 32
    alignas(128) __nv_bfloat16 w2[kMlpHidden * kMlpHidden];     // B, N = 64, K = 64
    alignas(16) float w3[kMlpHidden][8];                         // head (BF16 values), [in][out]
    float b1[kMlpHidden], b2[kMlpHidden], b3[kMlpOut];
    alignas(8) unsigned long long mbar;
    uint32_t tmem_base;
};

// two BF16 values at (row, k), (row, k + 1), k even: one 4-byte store
__device__ __forceinline__ void store_bf16x2(__nv_bfloat16 *base, uint32_t off, float lo,
                                             float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<unsigned char *>(base) + off) = h;
}

// BF16(max(lo, 0)) | BF16(max(hi, 0)) << 16, round to nearest even, in one
// conversion.  A NaN stays NaN (max(NaN, 0) would give 0): rows that can
// carry NaN features (zero quaternion, mean at the camera centre) are culled
// before their MLP outputs are used.
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// Loads the packed weights into canonical layout, initialises the mbarrier
// and allocates TMEM.  All threads of the CTA must call it.
__device__ __forceinline__ void setup(Smem &sm, const DevMLP &mlp) {
    for (int e = threadIdx.x; e < kMlpHidden * kMlpK1; e += blockDim.x) {
        const int n = e / kMlpK1, k = e % kMlpK1;
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(sm.w1) +
                                           core_off(n, k, kMlpK1)) = mlp.w1[e];
    }
    for (int e = threadIdx.x; e < kMlpHidden * kMlpHidden; e += blockDim.x) {
        const int n = e / kMlpHidden, k = e % kMlpHidden;
        *reinterpret_cast<__nv_bfloat16 *>(reinterpret_cast<unsigned char *>(sm.w2) +
                                           core_off(n, k, kMlpHidden)) = mlp.w2[e];
    }
    for (int e = threadIdx.x; e < kMlpHidden * 8; e += blockDim.x) {
        const int c = e >> 3, k = e & 7;
        sm.w3[c][k] = k < kMlpOut ? __bfloat162float(mlp.w3[k * kMlpHidden + c]) : 0.0f;
    }
    for (int e = threadIdx.x; e < kMlpHidden; e += blockDim.x) {
        sm.b1[e] = mlp.b1[e];
        sm.b2[e] = mlp.b2[e];
    }
    if (threadIdx.x < kMlpOut) sm.b3[threadIdx.x] = mlp.b3[threadIdx.x];
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&sm.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(&sm.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

__device__ __forceinline__ void teardown(Smem &sm) {
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem_base),
                     "r"(kTmemCols)
                     : "memory");
}

// Issues one layer (all K steps, both tiles) from thread 0 and waits for it.
// Tile t reads A at a_t and writes TMEM columns 64 t .. 64 t + 63.
__device__ __forceinline__ bool layer(Smem &sm, const void *a0, const void *a1, const void *b,
                                      int K, uint32_t &phase) {
    if (threadIdx.x == 0) {
        fence_after();
        const uint32_t sbo = (uint32_t)(K >> 3) << 7;
        const uint32_t idesc = idesc_bf16(kRows, kMlpHidden);
        const void *as[2] = {a0, a1};
#pragma unroll
        for (int t = 0; t < kTiles; ++t) {
#pragma unroll 1
            for (int s = 0; s < K / 16; ++s) {
                const uint64_t ad = smem_desc(saddr(as[t]) + (uint32_t)s * 256u, 128u, sbo);
                const uint64_t bd = smem_desc(saddr(b) + (uint32_t)s * 256u, 128u, sbo);
                mma(sm.tmem_base + 64u * (uint32_t)t, ad, bd, idesc, s > 0 ? 1u : 0u);
            }
        }
        commit(saddr(&sm.mbar));
    }
    const bool ok = wait(saddr(&sm.mbar), phase);
    phase ^= 1u;
    fence_after();
    return ok;
}

// Writes this thread's 32 features (tile threadIdx.x / 128, row
// threadIdx.x % 128) into the layer-1 operand as BF16.
__device__ __forceinline__ void put_features(Smem &sm, const float (&f)[kMlpK1]) {
    const int tile = threadIdx.x / kRows, row = threadIdx.x % kRows;
#pragma unroll
    for (int k = 0; k < kMlpK1; k += 2)
        store_bf16x2(sm.x[tile], core_off(row, k, kMlpK1), f[k], f[k + 1]);
}

// The MLP of the CTA's 256 rows: each thread has already written its row's
// 32 BF16 features into sm.x (put_features); out receives (phi-logit,
// o-logit, d_r, d_g, d_b) of its own row, biases added.  All threads call it.
__device__ __forceinline__ bool mlp_cta(Smem &sm, uint32_t &phase, float (&out)[5]) {
    const int tile = threadIdx.x / kRows, row = threadIdx.x % kRows;
    const int quad = (threadIdx.x >> 5) & 3;   // TMEM lane quadrant of this warp
    const uint32_t col0 = sm.tmem_base + 64u * (uint32_t)tile + ((uint32_t)(32 * quad) << 16);
    bool ok = true;
    fence_async_smem();
    fence_before();
    __syncthreads();
    // layer 1: [128 x 32] x [32 x 64] per tile
    ok &= layer(sm, sm.x[0], sm.x[1], sm.w1, kMlpK1, phase);
#pragma unroll
    for (int c = 0; c < kMlpHidden; c += 16) {
        float v[16];
        ld16(col0 + (uint32_t)c, v);
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
            uint4 u;
            u.x = relu_bf16x2(v[h] + sm.b1[c + h], v[h + 1] + sm.b1[c + h + 1]);
            u.y = relu_bf16x2(v[h + 2] + sm.b1[c + h + 2], v[h + 3] + sm.b1[c + h + 3]);
            u.z = relu_bf16x2(v[h + 4] + sm.b1[c + h + 4], v[h + 5] + sm.b1[c + h + 5]);
            u.w = relu_bf16x2(v[h + 6] + sm.b1[c + h + 6], v[h + 7] + sm.b1[c + h + 7]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(sm.h1[tile]) +
                                       core_off(row, c + h, kMlpHidden)) = u;
        }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    // layer 2: [128 x 64] x [64 x 64] per tile, into the same TMEM columns
    ok &= layer(sm, sm.h1[0], sm.h1[1], sm.w2, kMlpHidden, phase);
    float acc[kMlpOut];
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) acc[k] = sm.b3[k];
#pragma unroll
    for (int c = 0; c < kMlpHidden; c += 16) {
        float v[16];
        ld16(col0 + (uint32_t)c, v);
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
            // h2 = BF16(ReLU(.)), the same rounding the head MMA would see
            const uint32_t hp = relu_bf16x2(v[i] + sm.b2[c + i], v[i + 1] + sm.b2[c + i + 1]);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float h = j ? bf16_hi(hp) : bf16_lo(hp);
                const float4 w = *reinterpret_cast<const float4 *>(&sm.w3[c + i + j][0]);
                const float w4 = sm.w3[c + i + j][4];
                acc[0] = fmaf(w.x, h, acc[0]);
                acc[1] = fmaf(w.y, h, acc[1]);
                acc[2] = fmaf(w.z, h, acc[2]);
                acc[3] = fmaf(w.w, h, acc[3]);
                acc[4] = fmaf(w4, h, acc[4]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) out[k] = acc[k];
    fence_before();
    __syncthreads();
    return ok;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// The paper-width MLP_f (App. C: three hidden layers, e.g. 256, 128, 64):
// one CTA of 256 threads evaluates 256 Gaussians per step as two M = 128
// tiles, one after the other; layer l of a tile is one M = 128, N = h_l
// tcgen05 MMA chain (K = 16 per instruction) whose FP32 accumulator occupies
// TMEM columns 0 .. h_l - 1 (256 columns allocated).  All eight warps read
// each accumulator back: warps w and w + 4 share TMEM lanes 32 (w % 4).. and
// split the columns; each adds the bias, applies ReLU, rounds to BF16 and
// writes the next layer's A operand.  The 5-wide head runs on CUDA cores, the
// two halves' partial sums meeting in shared memory at the row's owner.
namespace tcw {

constexpr int kRows = 128;                    // rows per MMA tile
constexpr int kTiles = 2;                     // tiles per step, evaluated one after the other
constexpr int kThreads = kRows * kTiles;      // thread t owns row t % 128 of tile t / 128
constexpr int kTmemCols = 256;
constexpr uint32_t kXTileBytes = kRows * kMlpK1 * 2;

// Columns [lo, hi) of an N-column layer read back by warp half `half`
// (warps 0-3 or 4-7; warps w and w + 4 see the same TMEM lane quadrant), in
// units of 16 columns.
__device__ __forceinline__ void col_range(int N, int half, int &lo, int &hi) {
    const int u0 = ((N >> 4) + 1) >> 1;
    lo = half ? 16 * u0 : 0;
    hi = half ? N : 16 * u0;
}

__device__ __forceinline__ void put_bf16(unsigned char *base, uint32_t off, int row, int k, int K,
                                         __nv_bfloat16 v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off + tc::core_off(row, k, K)) = v;
}

__device__ __forceinline__ void setup(unsigned char *base, const WideLayout &L, const DevMLP &mlp) {
    const int h1 = mlp.h1, h2 = mlp.h2, h3 = mlp.h3;
    for (int e = threadIdx.x; e < h1 * kMlpK1; e += blockDim.x)
        put_bf16(base, L.w1, e / kMlpK1, e % kMlpK1, kMlpK1, mlp.w1[e]);
    for (int e = threadIdx.x; e < h2 * h1; e += blockDim.x)
        put_bf16(base, L.w2, e / h1, e % h1, h1, mlp.w2[e]);
    for (int e = threadIdx.x; e < h3 * h2; e += blockDim.x)
        put_bf16(base, L.w3, e / h2, e % h2, h2, mlp.w3[e]);
    float *head = reinterpret_cast<float *>(base + L.head);   // [h3][8]: input-major
    for (int e = threadIdx.x; e < h3 * 8; e += blockDim.x) {
        const int c = e >> 3, k = e & 7;
        head[e] = k < kMlpOut ? __bfloat162float(mlp.w4[k * h3 + c]) : 0.0f;
    }
    float *b1 = reinterpret_cast<float *>(base + L.b1);
    float *b2 = reinterpret_cast<float *>(base + L.b2);
    float *b3 = reinterpret_cast<float *>(base + L.b3);
    float *b4 = reinterpret_cast<float *>(base + L.b4);
    for (int e = threadIdx.x; e < h1; e += blockDim.x) b1[e] = mlp.b1[e];
    for (int e = threadIdx.x; e < h2; e += blockDim.x) b2[e] = mlp.b2[e];
    for (int e = threadIdx.x; e < h3; e += blockDim.x) b3[e] = mlp.b3[e];
    if (threadIdx.x < kMlpOut) b4[threadIdx.x] = mlp.b4[threadIdx.x];
    const uint32_t mbar = tc::saddr(base + L.mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::saddr(base + L.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

__device__ __forceinline__ void teardown(unsigned char *base, const WideLayout &L) {
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) {
        const uint32_t tmem = *reinterpret_cast<const uint32_t *>(base + L.tmem);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// D[128 x N] (TMEM columns 0..N-1) = A[128 x K] B[N x K]^T, issued by thread 0.
__device__ __forceinline__ bool layer(unsigned char *base, const WideLayout &L, uint32_t a_off,
                                      uint32_t b_off, int K, int N, uint32_t &phase) {
    const uint32_t tmem = *reinterpret_cast<const uint32_t *>(base + L.tmem);
    const uint32_t mbar = tc::saddr(base + L.mbar);
    if (threadIdx.x == 0) {
        tc::fence_after();
        const uint32_t sbo = (uint32_t)(K >> 3) << 7;
        const uint32_t idesc = tc::idesc_bf16(128, N);
        const uint32_t a0 = tc::saddr(base + a_off), b0 = tc::saddr(base + b_off);
#pragma unroll 1
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = tc::smem_desc(a0 + (uint32_t)s * 256u, 128u, sbo);
            const uint64_t bd = tc::smem_desc(b0 + (uint32_t)s * 256u, 128u, sbo);
            tc::mma(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc::commit(mbar);
    }
    const bool ok = tc::wait(mbar, phase);
    phase ^= 1u;
    tc::fence_after();
    return ok;
}

// BF16(ReLU(D + b)) into the next A operand (K = N): this thread's row
// (32 (warp % 4) + lane) and its warp half's columns; 64 columns per TMEM
// wait, each 8-column core-matrix row one 16-byte store.
__device__ __forceinline__ void relu_to_bf16(unsigned char *base, const WideLayout &L,
                                             uint32_t bias_off, uint32_t out_off, int N) {
    const int warp = threadIdx.x >> 5;
    const uint32_t tmem = *reinterpret_cast<const uint32_t *>(base + L.tmem);
    const uint32_t lane0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const float *b = reinterpret_cast<const float *>(base + bias_off);
    const int row = 32 * (warp & 3) + (threadIdx.x & 31);
    int lo, hi;
    col_range(N, warp >> 2, lo, hi);
#pragma unroll 1
    for (int c0 = lo; c0 < hi; c0 += 64) {
        uint32_t r[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + 16 * q < hi) tc::ld16_nowait(lane0 + (uint32_t)(c0 + 16 * q), r[q]);
        tc::ld_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (c0 + 16 * q >= hi) break;
#pragma unroll
            for (int h = 0; h < 16; h += 8) {
                const int c = c0 + 16 * q + h;
                uint4 u;
                uint32_t *w = &u.x;
#pragma unroll
                for (int i = 0; i < 8; i += 2)
                    w[i / 2] = tc::relu_bf16x2(__uint_as_float(r[q][h + i]) + b[c + i],
                                               __uint_as_float(r[q][h + i + 1]) + b[c + i + 1]);
                *reinterpret_cast<uint4 *>(base + out_off + tc::core_off(row, c, N)) = u;
            }
        }
    }
}

// Writes this thread's 32 features (tile threadIdx.x / 128, row
// threadIdx.x % 128) as BF16.
__device__ __forceinline__ void put_features(unsigned char *base, const WideLayout &L,
                                             const float (&f)[kMlpK1]) {
    __nv_bfloat16 *x = reinterpret_cast<__nv_bfloat16 *>(base + L.x + (threadIdx.x / kRows) * kXTileBytes);
#pragma unroll
    for (int k = 0; k < kMlpK1; k += 2)
        tc::store_bf16x2(x, tc::core_off(threadIdx.x % kRows, k, kMlpK1), f[k], f[k + 1]);
}

// The MLP of the step's two tiles, one after the other, every warp reading
// back its half of each layer's columns.  out = (phi-logit, o-logit, d_r,
// d_g, d_b) of the thread's own row (tile threadIdx.x / 128), biases added.
// All threads call it.
__device__ __forceinline__ bool mlp_cta(unsigned char *base, const WideLayout &L, int h1, int h2,
                                        int h3, uint32_t &phase, float (&out)[5]) {
    bool ok = true;
    const int warp = threadIdx.x >> 5, half = warp >> 2;
    const int row = 32 * (warp & 3) + (threadIdx.x & 31);
    const uint32_t tmem = *reinterpret_cast<const uint32_t *>(base + L.tmem);
    const uint32_t lane0 = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const float *b3 = reinterpret_cast<const float *>(base + L.b3);
    const float *head = reinterpret_cast<const float *>(base + L.head);
    const float *b4 = reinterpret_cast<const float *>(base + L.b4);
    float *red = reinterpret_cast<float *>(base + L.red) + row * 8;
    int lo3, hi3;
    col_range(h3, half, lo3, hi3);
#pragma unroll 1
    for (int t = 0; t < kTiles; ++t) {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        ok &= layer(base, L, L.x + (uint32_t)t * kXTileBytes, L.w1, kMlpK1, h1, phase);
        relu_to_bf16(base, L, L.b1, L.a0, h1);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        ok &= layer(base, L, L.a0, L.w2, h1, h2, phase);
        relu_to_bf16(base, L, L.b2, L.a1, h2);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        ok &= layer(base, L, L.a1, L.w3, h2, h3, phase);
        // third hidden layer BF16(ReLU(.)) in registers, then this half's
        // share of the head; the row's owner (warp half t) adds the other's
        float acc[kMlpOut] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int c0 = lo3; c0 < hi3; c0 += 64) {
            uint32_t r[4][16];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + 16 * q < hi3) tc::ld16_nowait(lane0 + (uint32_t)(c0 + 16 * q), r[q]);
            tc::ld_wait();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (c0 + 16 * q >= hi3) break;
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int c = c0 + 16 * q + i;
                    const uint32_t hp = tc::relu_bf16x2(__uint_as_float(r[q][i]) + b3[c],
                                                        __uint_as_float(r[q][i + 1]) + b3[c + 1]);
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const float h = j ? tc::bf16_hi(hp) : tc::bf16_lo(hp);
                        const float4 w = *reinterpret_cast<const float4 *>(head + (c + j) * 8);
                        const float w4 = head[(c + j) * 8 + 4];
                        acc[0] = fmaf(w.x, h, acc[0]);
                        acc[1] = fmaf(w.y, h, acc[1]);
                        acc[2] = fmaf(w.z, h, acc[2]);
                        acc[3] = fmaf(w.w, h, acc[3]);
                        acc[4] = fmaf(w4, h, acc[4]);
                    }
                }
            }
        }
        if (half != t) {
#pragma unroll
            for (int k = 0; k < kMlpOut; ++k) red[k] = acc[k];
        }
        tc::fence_before();
        __syncthreads();
        if (half == t) {
#pragma unroll
            for (int k = 0; k < kMlpOut; ++k) out[k] = b4[k] + acc[k] + red[k];
        }
    }
    tc::fence_before();
    __syncthreads();
    return ok;
}

}  // namespace tcw
}  // namespace mgs
