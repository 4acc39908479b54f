// Eq. 4 MLP on the tensor cores (shared by the forward preprocessing and the
// backward pass, which recomputes the hidden activations exactly as the
// forward produced them).
#pragma once

#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kMlpThreads = 128;  // 4 warps; each warp runs the MLP on 32 rows

// ---------------------------------------------------------------------------
// Eq. 4 on the tensor cores: mma.sync m16n8k16, BF16 inputs, FP32 accumulate.
// One warp evaluates 32 rows (its 32 Gaussians): rows 0-15 and 16-31 are two
// M tiles.  Layer-1 accumulators are reused in registers as layer-2 A
// fragments (same thread/element mapping), so hidden activations never leave
// the register file.
// ---------------------------------------------------------------------------

constexpr int kXStride = 40;   // bf16 per feature row in shared memory (80 B)
constexpr int kW1Stride = 40;  // bf16 per W1 row (80 B): conflict-free B loads
constexpr int kW2Stride = 72;  // bf16 per W2/W3 row (144 B)

struct MlpSmem {
    __nv_bfloat16 w1[kMlpHidden * kW1Stride];
    __nv_bfloat16 w2[kMlpHidden * kW2Stride];
    __nv_bfloat16 w3[kMlpN3 * kW2Stride];
    float b1[kMlpHidden];
    float b2[kMlpHidden];
    float b3[kMlpN3];
    __nv_bfloat16 x[kMlpThreads / 32][32 * kXStride];
    float out[kMlpThreads / 32][32][kMlpN3];
};

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

constexpr int kHStride = 72;   // bf16 per kept hidden row (144 B)

// Writes the packed hidden fragments h[4][4] (see mlp_warp) of rows r0, r1.
__device__ __forceinline__ void store_hidden(const uint32_t (&h)[4][4], __nv_bfloat16 *dst,
                                             int r0, int r1, int t) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        *reinterpret_cast<uint32_t *>(&dst[r0 * kHStride + 16 * j + 2 * t]) = h[j][0];
        *reinterpret_cast<uint32_t *>(&dst[r1 * kHStride + 16 * j + 2 * t]) = h[j][1];
        *reinterpret_cast<uint32_t *>(&dst[r0 * kHStride + 16 * j + 8 + 2 * t]) = h[j][2];
        *reinterpret_cast<uint32_t *>(&dst[r1 * kHStride + 16 * j + 8 + 2 * t]) = h[j][3];
    }
}

__device__ void mlp_load_weights(MlpSmem &sm, const DevMLP &mlp) {
    for (int k = threadIdx.x; k < kMlpHidden * kMlpK1 / 2; k += blockDim.x) {
        int r = k / (kMlpK1 / 2), c = 2 * (k % (kMlpK1 / 2));
        *reinterpret_cast<uint32_t *>(&sm.w1[r * kW1Stride + c]) =
            *reinterpret_cast<const uint32_t *>(&mlp.w1[r * kMlpK1 + c]);
    }
    for (int k = threadIdx.x; k < kMlpHidden * kMlpHidden / 2; k += blockDim.x) {
        int r = k / (kMlpHidden / 2), c = 2 * (k % (kMlpHidden / 2));
        *reinterpret_cast<uint32_t *>(&sm.w2[r * kW2Stride + c]) =
            *reinterpret_cast<const uint32_t *>(&mlp.w2[r * kMlpHidden + c]);
    }
    for (int k = threadIdx.x; k < kMlpN3 * kMlpHidden / 2; k += blockDim.x) {
        int r = k / (kMlpHidden / 2), c = 2 * (k % (kMlpHidden / 2));
        *reinterpret_cast<uint32_t *>(&sm.w3[r * kW2Stride + c]) =
            *reinterpret_cast<const uint32_t *>(&mlp.w3[r * kMlpHidden + c]);
    }
    for (int k = threadIdx.x; k < kMlpHidden; k += blockDim.x) {
        sm.b1[k] = mlp.b1[k];
        sm.b2[k] = mlp.b2[k];
    }
    if (threadIdx.x < kMlpN3) sm.b3[threadIdx.x] = mlp.b3[threadIdx.x];
}

// Runs the MLP on the 32 feature rows of this warp; row r's five outputs land
// in sm.out[warp][r][0..4].  kKeep: also store the BF16 hidden activations
// h1, h2 of row r at h1s[r * kHStride ..], h2s[r * kHStride ..].
template <bool kKeep>
__device__ __forceinline__ void mlp_warp(MlpSmem &sm, int warp, int lane, __nv_bfloat16 *h1s,
                                         __nv_bfloat16 *h2s) {
    const int g = lane >> 2, t = lane & 3;
    const __nv_bfloat16 *X = sm.x[warp];
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        // layer 1: [16 x 32] x [32 x 64]
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t a[4];
            a[0] = lds32(&X[r0 * kXStride + ks * 16 + 2 * t]);
            a[1] = lds32(&X[r1 * kXStride + ks * 16 + 2 * t]);
            a[2] = lds32(&X[r0 * kXStride + ks * 16 + 2 * t + 8]);
            a[3] = lds32(&X[r1 * kXStride + ks * 16 + 2 * t + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16 *wr = &sm.w1[(nt * 8 + g) * kW1Stride + ks * 16 + 2 * t];
                mma16816(acc[nt], a, lds32(wr), lds32(wr + 8));
            }
        }
        uint32_t h[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int nt = 2 * j + hh;
                const float bl = sm.b1[nt * 8 + 2 * t], bh = sm.b1[nt * 8 + 2 * t + 1];
                h[j][2 * hh] = pack_bf16(fmaxf(acc[nt][0] + bl, 0.f), fmaxf(acc[nt][1] + bh, 0.f));
                h[j][2 * hh + 1] =
                    pack_bf16(fmaxf(acc[nt][2] + bl, 0.f), fmaxf(acc[nt][3] + bh, 0.f));
            }
        }
        // h[j] is the layer-2 A fragment of k-step j: (row g, k lo), (row g+8, k lo),
        // (row g, k hi), (row g+8, k hi) -- exactly the accumulator layout of
        // n-tiles 2j and 2j+1.
        if constexpr (kKeep) store_hidden(h, h1s, r0, r1, t);
        // layer 2: [16 x 64] x [64 x 64]
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const __nv_bfloat16 *wr = &sm.w2[(nt * 8 + g) * kW2Stride + ks * 16 + 2 * t];
                mma16816(acc[nt], h[ks], lds32(wr), lds32(wr + 8));
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int nt = 2 * j + hh;
                const float bl = sm.b2[nt * 8 + 2 * t], bh = sm.b2[nt * 8 + 2 * t + 1];
                h[j][2 * hh] = pack_bf16(fmaxf(acc[nt][0] + bl, 0.f), fmaxf(acc[nt][1] + bh, 0.f));
                h[j][2 * hh + 1] =
                    pack_bf16(fmaxf(acc[nt][2] + bl, 0.f), fmaxf(acc[nt][3] + bh, 0.f));
            }
        }
        if constexpr (kKeep) store_hidden(h, h2s, r0, r1, t);
        // head: [16 x 64] x [64 x 8]
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const __nv_bfloat16 *wr = &sm.w3[g * kW2Stride + ks * 16 + 2 * t];
            mma16816(o, h[ks], lds32(wr), lds32(wr + 8));
        }
        sm.out[warp][r0][2 * t] = o[0] + sm.b3[2 * t];
        sm.out[warp][r0][2 * t + 1] = o[1] + sm.b3[2 * t + 1];
        sm.out[warp][r1][2 * t] = o[2] + sm.b3[2 * t];
        sm.out[warp][r1][2 * t + 1] = o[3] + sm.b3[2 * t + 1];
    }
}


}  // namespace
}  // namespace mgs
