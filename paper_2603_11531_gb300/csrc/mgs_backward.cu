// Backward pass: the adjoint of the forward render (Sec. 3.1 Eq. 2-4, Sec. 3.2,
// App. B), for training through torch.autograd.
//
// Per pixel p with C = (1 - T) A / B + T c_bg, r = A / B, G = dL/dC(p):
//   dL/dc_i  += (1 - T)/B * a_i w_i G
//   dL/dw_i  += (1 - T)/B * a_i G.(c_i - r)
//   dL/da_i  += w_i (1 - T)/B G.(c_i - r) - T/(1 - a_i) G.(c_bg - r)
// and through a_i = o_i exp(-q/2) (zero when the 0.99 clamp is active) to
// o_i, the pixel mean and the conic.  All of these only need (A, B, T) of the
// forward, so the backward is as order-independent as the forward.
//
//   k_raster_bwd      one CTA per tile, same blocks and culling as the
//                     forward; per-Gaussian partials are reduced across the
//                     warp and added to a per-Gaussian gradient record.
//   k_preprocess_bwd  one thread per Gaussian: recomputes the forward, chains
//                     through the EWA covariance, projection, SH colour,
//                     Eq. 3 weight and (warp-cooperatively) the Eq. 4 MLP.
//                     The MLP's deltas and weight gradients are TF32 mma.sync
//                     products (FP32 accumulation); weight gradients stay in
//                     registers across the CTA's rows, are written once per
//                     CTA and reduced in a fixed order by k_mlp_grad_reduce.
#include "mgs_internal.cuh"
#include "mgs_mlp.cuh"

namespace mgs {
namespace {

constexpr int kBwdThreads = 64;   // raster backward: two warps per tile
constexpr int kRedGroup = 8;      // candidates reduced together through shared memory
constexpr int kGRec = 12;         // per-Gaussian raster gradient record
// layout: dc(3), dw, do, dm(2), dK(3) [conic A, B, C], pad(2)

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kBwdThreads) k_raster_bwd(RenderArgs args,
                                                            const float *__restrict__ dL,
                                                            const float *__restrict__ aux,
                                                            float *__restrict__ gG) {
    __shared__ float4 buf[2][4][32];
    // per warp: the partials of up to kRedGroup candidates, row (k, e), column
    // lane; rows padded to 36 floats so eight lanes reading eight rows with
    // 16-byte loads hit distinct banks
    __shared__ __align__(16) float red[2][kRedGroup * 10][36];
    const DevCamera &cam = args.cam;
    const int tile = (int)(args.tile_order[blockIdx.x] & kTileMask);
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile, by0 = ty * kTile + 8 * warp;
    const int px0 = bx0 + 4 * (lane & 3);
    const int py = by0 + (lane >> 2);
    if (args.status->last_pairs > args.capacity) return;

    // per-pixel constants from the forward's (A, B, T) and dL/dC, with
    // k_A = (1 - T) / B and r = A / B:  kG = k_A G,  kGr = k_A G.r,
    // TGb = T G.(c_bg - r)  (all zero for pixels without coverage)
    const int64_t HW = (int64_t)cam.width * cam.height;
    float kG[4][3], kGr[4], TGb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = px0 + k;
        kG[k][0] = kG[k][1] = kG[k][2] = kGr[k] = TGb[k] = 0.f;
        if (x < cam.width && py < cam.height) {
            const int64_t p = (int64_t)py * cam.width + x;
            const float B = aux[3 * HW + p];
            if (B > 0.0f) {
                const float T = aux[4 * HW + p];
                const float inv = 1.0f / B;
                const float kA = (1.0f - T) * inv;
                float G[3], r[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    G[ch] = dL[3 * p + ch];
                    r[ch] = aux[ch * HW + p] * inv;
                    kG[k][ch] = kA * G[ch];
                }
                kGr[k] = kA * (G[0] * r[0] + G[1] * r[1] + G[2] * r[2]);
                TGb[k] = T * (G[0] * (args.bg[0] - r[0]) + G[1] * (args.bg[1] - r[1]) +
                              G[2] * (args.bg[2] - r[2]));
            }
        }
    }
    const uint32_t start = args.tile_offsets[tile];
    const uint32_t end = args.tile_offsets[tile + 1];
    const float bx = (float)bx0 + 8.0f, by = (float)by0 + 4.0f;
    const float pyc = (float)py + 0.5f;
    const float kq = -0.72134752044448170f;  // -log2(e) / 2
    float4(*wb)[32] = buf[warp];

    // list entries two batches ahead, their records one batch ahead
    uint32_t gid_n = 0, gid_nn = 0;
    float4 a_n = make_float4(0.f, 0.f, 0.f, 0.f), b_n = a_n, c_n = a_n;
    if (start + lane < end) {
        gid_n = __ldg(&args.gids[start + lane]);
        a_n = __ldg(&args.rec[gid_n].a);
        b_n = __ldg(&args.rec[gid_n].b);
        c_n = __ldg(&args.rec[gid_n].c);
    }
    if (start + 32 + lane < end) gid_nn = __ldg(&args.gids[start + 32 + lane]);
    for (uint32_t base = start; base < end; base += 32) {
        const uint32_t j = base + lane;
        const uint32_t gid = gid_n;
        const float4 a = a_n, b = b_n, c = c_n;
        const bool cand = j < end && block_may_hit(a.x, a.y, a.z, a.w, b.x, bx, by, 7.5f, 3.5f);
        if (j + 32 < end) {
            gid_n = gid_nn;
            a_n = __ldg(&args.rec[gid_n].a);
            b_n = __ldg(&args.rec[gid_n].b);
            c_n = __ldg(&args.rec[gid_n].c);
        }
        if (j + 64 < end) gid_nn = __ldg(&args.gids[j + 64]);
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (cand) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            const float w = -b.z, o = exp2f(b.y);
            const float iw = 1.0f / w;
            wb[0][pos] = a;
            // 1/o (0 when o = 0: no opacity gradient then)
            wb[1][pos] = make_float4(b.x, b.y, o > 0.0f ? 1.0f / o : 0.0f, w);
            // colour c = (-w c) / (-w); conic (A, B, C) = L L^T from the factors
            wb[2][pos] = make_float4(-b.w * iw, -c.x * iw, -c.y * iw, a.z * a.z);
            wb[3][pos] = make_float4(a.z * a.w, a.w * a.w + b.x * b.x, __uint_as_float(gid), 0.f);
        }
        __syncwarp();
        const int nc = __popc(bal);
        for (int k0 = 0; k0 < nc; k0 += kRedGroup) {
        const int ng = min(kRedGroup, nc - k0);
        for (int k = k0; k < k0 + ng; ++k) {
            const float4 cs0 = wb[0][k], cs1 = wb[1][k], cs2 = wb[2][k], cs3 = wb[3][k];
            const float mx = cs0.x, my = cs0.y, l11 = cs0.z, l21 = cs0.w;
            const float l22 = cs1.x, lo = cs1.y, io = cs1.z, w = cs1.w;
            const float cr = cs2.x, cg = cs2.y, cb = cs2.z, cA = cs2.w, cB = cs3.x, cC = cs3.y;
            // per pixel with q <= 9 (a = min(a_raw, 0.99), u = k_A (G.c - G.r)):
            //   dc  += w a kG          dw += a u
            // and, where the clamp is inactive, with s = a (w u - TGb / (1 - a)):
            //   do  += s / o,  and s, s dx, s dx^2 for the mean and conic terms
            // (dy is the same for the lane's four pixels)
            float sc0 = 0.f, sc1 = 0.f, sc2 = 0.f, sw = 0.f;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            const float dy = __fsub_rn(pyc, my);
            const float ldy = __fmul_rn(l21, dy);
            const float e2 = __fmul_rn(l22, dy);
            const float e2s = __fmul_rn(e2, e2);
#pragma unroll
            for (int px = 0; px < 4; ++px) {
                const float dx = __fsub_rn((float)(px0 + px) + 0.5f, mx);
                const float e1 = __fmaf_rn(l11, dx, ldy);
                const float q = __fmaf_rn(e1, e1, e2s);
                if (!(q <= 9.0f)) continue;
                const float araw = ex2f(__fmaf_rn(q, kq, lo));
                const float al = fminf(araw, 0.99f);
                sc0 = fmaf(al, kG[px][0], sc0);
                sc1 = fmaf(al, kG[px][1], sc1);
                sc2 = fmaf(al, kG[px][2], sc2);
                const float u = fmaf(kG[px][0], cr, fmaf(kG[px][1], cg, fmaf(kG[px][2], cb, -kGr[px])));
                sw = fmaf(al, u, sw);
                if (araw < 0.99f) {
                    // 1 - al > 0.01: the fast reciprocal division is accurate to a few ulp
                    const float sa = al * fmaf(w, u, -__fdividef(TGb[px], 1.0f - al));
                    s0 += sa;
                    s1 = fmaf(sa, dx, s1);
                    s2 = fmaf(sa * dx, dx, s2);
                }
            }
            float acc[10];
            acc[0] = w * sc0;
            acc[1] = w * sc1;
            acc[2] = w * sc2;
            acc[3] = sw;
            if (io > 0.0f) {
                // dL/dq = -s / 2 per pixel; q = A dx^2 + 2 B dx dy + C dy^2 gives
                // dq/dm = -2 (A dx + B dy, B dx + C dy) and dq/d(A, B, C) =
                // (dx^2, 2 dx dy, dy^2)
                acc[4] = s0 * io;
                acc[5] = fmaf(cA, s1, cB * dy * s0);
                acc[6] = fmaf(cB, s1, cC * dy * s0);
                acc[7] = -0.5f * s2;
                acc[8] = -dy * s1;
                acc[9] = -0.5f * dy * dy * s0;
            } else {
                acc[4] = acc[5] = acc[6] = acc[7] = acc[8] = acc[9] = 0.f;
            }
#pragma unroll
            for (int e = 0; e < 10; ++e) red[warp][(k - k0) * 10 + e][lane] = acc[e];
        }
        __syncwarp();
        // transposed reduction: lane r sums row r (one candidate's partial e over
        // the 32 lanes) and adds it to that candidate's gradient record
        for (int r = lane; r < ng * 10; r += 32) {
            const float4 *row = reinterpret_cast<const float4 *>(red[warp][r]);
            float sum = 0.f;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const float4 x = row[v];
                sum += (x.x + x.y) + (x.z + x.w);
            }
            if (sum != 0.0f) {
                const int k = k0 + r / 10;
                atomicAdd(gG + (size_t)__float_as_uint(wb[3][k].z) * kGRec + (r % 10), sum);
            }
        }
        __syncwarp();
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Preprocessing adjoint.
// ---------------------------------------------------------------------------

constexpr int kMlpGrad = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden +
                         kMlpHidden + kMlpOut * kMlpHidden + kMlpOut;  // 5957
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpHidden * kMlpIn, kOffW2 = kOffB1 + kMlpHidden,
              kOffB2 = kOffW2 + kMlpHidden * kMlpHidden, kOffW3 = kOffB2 + kMlpHidden,
              kOffB3 = kOffW3 + kMlpOut * kMlpHidden;

// Row buffers of the MLP adjoint hold the CTA's 128 rows (row = warp * 32 +
// lane).  Strides: 72 floats per delta row make the transposed fragment
// loads of the weight-gradient products conflict-free; 8 per d3 row and 24
// per staged dx row.
constexpr int kRows = kMlpThreads;
constexpr int kDS = 72;
constexpr int kD3S = 8;
constexpr int kDxS = 24;
constexpr int kOnesCol = kMlpHidden;  // h1 column 64 holds 1: its products give dL/db2
constexpr int kXOnesCol = kMlpIn;     // x column 22 holds 1: its products give dL/db1

// About 108 KB, two CTAs per SM: d1 overwrites d2 once the products that
// need d2 are done, and dx reuses h2's space once h2 is no longer read.
struct BwdSmem {
    MlpSmem mlp;                          // weights, BF16 features x, head outputs
    __nv_bfloat16 h1[kRows * kHStride];   // BF16 hidden activations (forward recompute)
    union {
        __nv_bfloat16 h2[kRows * kHStride];
        float dx[kRows * kDxS];           // dL/d(features), staged for the row threads
    };
    float dd[kRows * kDS];                // dL/d(pre-activation 2), then of pre-activation 1
    float d3[kRows * kD3S];               // dL/d(head outputs), columns 5..7 zero
    float b3[kMlpThreads / 32][8];        // per-warp sums of d3
};
static_assert(kRows * kDxS * sizeof(float) <= kRows * kHStride * sizeof(__nv_bfloat16),
              "dx fits in h2's space");

// Weight-gradient accumulators of one lane (m16n8 fragments): warp w owns
// rows 16w..16w+15 of dW2 (nine n-tiles, the last one the b2 column), of dW1
// (three n-tiles; column 22 is b1) and of dW3^T.
struct WGradAcc {
    float w2[9][4];
    float w1[3][4];
    float w3[4];
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// A BF16 value as a TF32 operand (exact: BF16 keeps 8 significand bits).
__device__ __forceinline__ uint32_t bf_tf32(const __nv_bfloat16 *p) {
    return (uint32_t)(*reinterpret_cast<const unsigned short *>(p)) << 16;
}
// D += A B, m16n8k8, TF32 operands, FP32 accumulation.  Fragments (g = lane / 4,
// t = lane % 4): a = A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4]; b = B[t][g],
// B[t+4][g]; d = D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1].
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float2 relu_mask(const __nv_bfloat16 *h, float a, float b) {
    const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(h);
    return make_float2(__low2float(m) > 0.0f ? a : 0.0f, __high2float(m) > 0.0f ? b : 0.0f);
}

// The adjoint of the Eq. 4 MLP for the CTA's 128 rows (d3 in shared memory)
// runs in four steps, with a CTA barrier after each of the first three:
//   1. mlp_d2_warp      d2 = (d3 W3) * [h2 > 0] for the warp's 32 rows;
//   2. mlp_wgrad2_cta   dW2 += d2^T [h1 | 1] and dW3^T += h2^T d3;
//   3. mlp_d1_warp      d1 = (d2 W2) * [h1 > 0] over d2 in place and
//                       dx = d1 W1 into h2's space, for the warp's rows;
//   4. mlp_wgrad1_cta   dW1 += d1^T [x | 1].
// TF32 products, FP32 accumulation.

__device__ __forceinline__ void mlp_d2_warp(BwdSmem &sm, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = warp * 32 + mt * 16 + g, r1 = r0 + 8;
        const uint32_t a0 = to_tf32(sm.d3[r0 * kD3S + t]), a1 = to_tf32(sm.d3[r1 * kD3S + t]);
        const uint32_t a2 = to_tf32(sm.d3[r0 * kD3S + t + 4]);
        const uint32_t a3 = to_tf32(sm.d3[r1 * kD3S + t + 4]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_tf32(c, a0, a1, a2, a3, bf_tf32(&sm.mlp.w3[t * kW2Stride + nt * 8 + g]),
                     bf_tf32(&sm.mlp.w3[(t + 4) * kW2Stride + nt * 8 + g]));
            const int col = nt * 8 + 2 * t;
            *reinterpret_cast<float2 *>(&sm.dd[r0 * kDS + col]) =
                relu_mask(&sm.h2[r0 * kHStride + col], c[0], c[1]);
            *reinterpret_cast<float2 *>(&sm.dd[r1 * kDS + col]) =
                relu_mask(&sm.h2[r1 * kHStride + col], c[2], c[3]);
        }
    }
}

// The d1 accumulators serve directly as the A fragments of dx = d1 W1,
// taking k = 2t and 2t + 1 of each step for fragment columns t and t + 4
// (B rows follow the same order).
__device__ __forceinline__ void mlp_d1_warp(BwdSmem &sm, int warp, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = warp * 32 + mt * 16 + g, r1 = r0 + 8;
        float c[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
            const int k0 = ks * 8;
            const uint32_t a0 = to_tf32(sm.dd[r0 * kDS + k0 + t]);
            const uint32_t a1 = to_tf32(sm.dd[r1 * kDS + k0 + t]);
            const uint32_t a2 = to_tf32(sm.dd[r0 * kDS + k0 + t + 4]);
            const uint32_t a3 = to_tf32(sm.dd[r1 * kDS + k0 + t + 4]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
                mma_tf32(c[nt], a0, a1, a2, a3, bf_tf32(&sm.mlp.w2[(k0 + t) * kW2Stride + nt * 8 + g]),
                         bf_tf32(&sm.mlp.w2[(k0 + t + 4) * kW2Stride + nt * 8 + g]));
        }
        __syncwarp();   // every lane has read this m-tile's d2 rows: overwrite them with d1
        float dx[3][4];
#pragma unroll
        for (int ft = 0; ft < 3; ++ft) dx[ft][0] = dx[ft][1] = dx[ft][2] = dx[ft][3] = 0.f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = nt * 8 + 2 * t;
            const float2 e0 = relu_mask(&sm.h1[r0 * kHStride + col], c[nt][0], c[nt][1]);
            const float2 e1 = relu_mask(&sm.h1[r1 * kHStride + col], c[nt][2], c[nt][3]);
            *reinterpret_cast<float2 *>(&sm.dd[r0 * kDS + col]) = e0;
            *reinterpret_cast<float2 *>(&sm.dd[r1 * kDS + col]) = e1;
            const uint32_t a0 = to_tf32(e0.x), a1 = to_tf32(e1.x), a2 = to_tf32(e0.y),
                           a3 = to_tf32(e1.y);
#pragma unroll
            for (int ft = 0; ft < 3; ++ft)
                mma_tf32(dx[ft], a0, a1, a2, a3, bf_tf32(&sm.mlp.w1[col * kW1Stride + ft * 8 + g]),
                         bf_tf32(&sm.mlp.w1[(col + 1) * kW1Stride + ft * 8 + g]));
        }
#pragma unroll
        for (int ft = 0; ft < 3; ++ft) {
            const int col = ft * 8 + 2 * t;
            *reinterpret_cast<float2 *>(&sm.dx[r0 * kDxS + col]) = make_float2(dx[ft][0], dx[ft][1]);
            *reinterpret_cast<float2 *>(&sm.dx[r1 * kDxS + col]) = make_float2(dx[ft][2], dx[ft][3]);
        }
    }
}

// Weight gradients of the CTA's 128 rows into this lane's accumulators, each
// a sum over the rows (the K dimension), warp w taking output rows
// 16w..16w+15.
__device__ __forceinline__ void mlp_wgrad2_cta(const BwdSmem &sm, int warp, int lane, WGradAcc &acc) {
    const int g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16 + g, m1 = m0 + 8;
#pragma unroll 2
    for (int ks = 0; ks < kRows / 8; ++ks) {
        const int ra = ks * 8 + t, rb = ra + 4;
        const uint32_t a0 = to_tf32(sm.dd[ra * kDS + m0]), a1 = to_tf32(sm.dd[ra * kDS + m1]);
        const uint32_t a2 = to_tf32(sm.dd[rb * kDS + m0]), a3 = to_tf32(sm.dd[rb * kDS + m1]);
#pragma unroll
        for (int nt = 0; nt < 9; ++nt)
            mma_tf32(acc.w2[nt], a0, a1, a2, a3, bf_tf32(&sm.h1[ra * kHStride + nt * 8 + g]),
                     bf_tf32(&sm.h1[rb * kHStride + nt * 8 + g]));
        mma_tf32(acc.w3, bf_tf32(&sm.h2[ra * kHStride + m0]), bf_tf32(&sm.h2[ra * kHStride + m1]),
                 bf_tf32(&sm.h2[rb * kHStride + m0]), bf_tf32(&sm.h2[rb * kHStride + m1]),
                 to_tf32(sm.d3[ra * kD3S + g]), to_tf32(sm.d3[rb * kD3S + g]));
    }
}

__device__ __forceinline__ void mlp_wgrad1_cta(const BwdSmem &sm, int warp, int lane, WGradAcc &acc) {
    const int g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16 + g, m1 = m0 + 8;
    const __nv_bfloat16 *X = &sm.mlp.x[0][0];
#pragma unroll 2
    for (int ks = 0; ks < kRows / 8; ++ks) {
        const int ra = ks * 8 + t, rb = ra + 4;
        const uint32_t a0 = to_tf32(sm.dd[ra * kDS + m0]), a1 = to_tf32(sm.dd[ra * kDS + m1]);
        const uint32_t a2 = to_tf32(sm.dd[rb * kDS + m0]), a3 = to_tf32(sm.dd[rb * kDS + m1]);
#pragma unroll
        for (int ft = 0; ft < 3; ++ft)
            mma_tf32(acc.w1[ft], a0, a1, a2, a3, bf_tf32(&X[ra * kXStride + ft * 8 + g]),
                     bf_tf32(&X[rb * kXStride + ft * 8 + g]));
    }
}

template <bool kFP16>
__device__ __forceinline__ void load_rec(const void *attrs, int64_t i, float (&v)[kRec]) {
    if constexpr (kFP16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(attrs) + 3 * i;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 u = __ldg(p + k);
            const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = __half22float2(h[j]);
                v[8 * k + 2 * j] = f.x;
                v[8 * k + 2 * j + 1] = f.y;
            }
        }
    } else {
        const float4 *p = reinterpret_cast<const float4 *>(attrs) + 6 * i;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 f = __ldg(p + k);
            v[4 * k] = f.x;
            v[4 * k + 1] = f.y;
            v[4 * k + 2] = f.z;
            v[4 * k + 3] = f.w;
        }
    }
}

template <bool kFP16, bool kMLP, bool kResidual>
__global__ void __launch_bounds__(kMlpThreads) k_preprocess_bwd(RenderArgs args,
                                                               const float *__restrict__ gG,
                                                               float *__restrict__ d_attrs,
                                                               float *__restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &sm = *reinterpret_cast<BwdSmem *>(smem_raw);
    const DevCamera &cam = args.cam;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (kMLP) {
        mlp_load_weights(sm.mlp, args.mlp);
        // h1 columns 64..71: a column of ones (bias gradient b2), then zeros
        for (int e = threadIdx.x; e < kRows * 8; e += blockDim.x)
            sm.h1[(e >> 3) * kHStride + kOnesCol + (e & 7)] =
                __float2bfloat16((e & 7) == 0 ? 1.0f : 0.0f);
    }
    WGradAcc wacc;
    float sb3[kMlpOut];
    if constexpr (kMLP) {
#pragma unroll
        for (int nt = 0; nt < 9; ++nt) wacc.w2[nt][0] = wacc.w2[nt][1] = wacc.w2[nt][2] = wacc.w2[nt][3] = 0.f;
#pragma unroll
        for (int ft = 0; ft < 3; ++ft) wacc.w1[ft][0] = wacc.w1[ft][1] = wacc.w1[ft][2] = wacc.w1[ft][3] = 0.f;
        wacc.w3[0] = wacc.w3[1] = wacc.w3[2] = wacc.w3[3] = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) sb3[k] = 0.f;
    }
    const float *W = cam.R;
    float cc[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) cc[j] = -(W[j] * cam.t[0] + W[3 + j] * cam.t[1] + W[6 + j] * cam.t[2]);
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float limx = 1.3f * (0.5f * (float)cam.width / cam.fx);
    const float limy = 1.3f * (0.5f * (float)cam.height / cam.fy);

    for (int64_t base = (int64_t)blockIdx.x * kMlpThreads; base < args.n;
         base += (int64_t)gridDim.x * kMlpThreads) {
        // the previous iteration's weight-gradient products read every warp's rows
        if constexpr (kMLP) __syncthreads();
        const int64_t i = base + threadIdx.x;
        const bool valid = i < args.n;
        float v[kRec];
#pragma unroll
        for (int k = 0; k < kRec; ++k) v[k] = 0.f;
        bool vis = false;
        if (valid) {
            load_rec<kFP16>(args.attrs, i, v);
            const uint2 r = args.rect[i];
            vis = (r.x != 0u || r.y != 0u) && ((r.x >> 16) > (r.x & 0xFFFF));
        }
        float up[10];
#pragma unroll
        for (int e = 0; e < 10; ++e) up[e] = vis ? gG[(size_t)i * kGRec + e] : 0.f;
        // ---- forward recompute (FP32) ----
        const float qn = sqrtf(v[6] * v[6] + v[7] * v[7] + v[8] * v[8] + v[9] * v[9]);
        const float iqn = vis ? 1.0f / qn : 0.f;
        const float qw = v[6] * iqn, qx = v[7] * iqn, qy = v[8] * iqn, qz = v[9] * iqn;
        float d[3] = {v[0] - cc[0], v[1] - cc[1], v[2] - cc[2]};
        const float dn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const float idn = dn > 0.f ? 1.0f / dn : 0.f;
        const float P[3] = {d[0] * idn, d[1] * idn, d[2] * idn};

        float phi = 1.0f, o = v[10], yv[5] = {1.f, 0.f, 0.f, 0.f, 0.f};
        if constexpr (kMLP) {
            __nv_bfloat16 *xr = &sm.mlp.x[warp][lane * kXStride];
            float f[kMlpK1];
#pragma unroll
            for (int k = 0; k < kMlpK1; ++k) f[k] = 0.f;
            if (valid) {
                f[0] = P[0]; f[1] = P[1]; f[2] = P[2];
                f[3] = v[3]; f[4] = v[4]; f[5] = v[5];
                f[6] = qw; f[7] = qx; f[8] = qy; f[9] = qz;
#pragma unroll
                for (int k = 0; k < 12; ++k) f[10 + k] = v[11 + k];
            }
            f[kXOnesCol] = 1.0f;  // W1's column 22 is zero: the forward is unchanged
#pragma unroll
            for (int k = 0; k < kMlpK1; k += 8) {
                uint4 u;
                u.x = pack_bf16(f[k], f[k + 1]);
                u.y = pack_bf16(f[k + 2], f[k + 3]);
                u.z = pack_bf16(f[k + 4], f[k + 5]);
                u.w = pack_bf16(f[k + 6], f[k + 7]);
                *reinterpret_cast<uint4 *>(xr + k) = u;
            }
            __syncwarp();
            mlp_warp<true>(sm.mlp, warp, lane, sm.h1 + warp * 32 * kHStride, sm.h2 + warp * 32 * kHStride);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 5; ++k) yv[k] = sm.mlp.out[warp][lane][k];
            phi = fmaxf(yv[0], 0.f);
            o = 1.0f / (1.0f + __expf(-yv[1]));
        }
        // colour
        float cbase[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            cbase[ch] = C0 * v[11 + ch] - C1 * P[1] * v[14 + ch] + C1 * P[2] * v[17 + ch] -
                       C1 * P[0] * v[20 + ch] + 0.5f;
            if constexpr (kResidual) cbase[ch] += yv[2 + ch];
        }
        // projection
        float R[9];
        R[0] = 1.f - 2.f * (qy * qy + qz * qz);
        R[1] = 2.f * (qx * qy - qw * qz);
        R[2] = 2.f * (qx * qz + qw * qy);
        R[3] = 2.f * (qx * qy + qw * qz);
        R[4] = 1.f - 2.f * (qx * qx + qz * qz);
        R[5] = 2.f * (qy * qz - qw * qx);
        R[6] = 2.f * (qx * qz - qw * qy);
        R[7] = 2.f * (qy * qz + qw * qx);
        R[8] = 1.f - 2.f * (qx * qx + qy * qy);
        float t[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) t[r] = W[3 * r] * v[0] + W[3 * r + 1] * v[1] + W[3 * r + 2] * v[2] + cam.t[r];
        const float rz = vis ? 1.0f / t[2] : 0.f;
        const float u = t[0] * rz, vv = t[1] * rz;
        const bool cx_ = fabsf(u) > limx, cy_ = fabsf(vv) > limy;
        const float uc = fminf(fmaxf(u, -limx), limx), vc = fminf(fmaxf(vv, -limy), limy);
        const float J00 = cam.fx * rz, J02 = -cam.fx * uc * rz;
        const float J11 = cam.fy * rz, J12 = -cam.fy * vc * rz;
        float T0[3], T1[3], M[9], V0[3], V1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T0[j] = J00 * W[j] + J02 * W[6 + j];
            T1[j] = J11 * W[3 + j] + J12 * W[6 + j];
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) M[3 * k + j] = R[3 * k + j] * v[3 + j];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            V0[j] = T0[0] * M[j] + T0[1] * M[3 + j] + T0[2] * M[6 + j];
            V1[j] = T1[0] * M[j] + T1[1] * M[3 + j] + T1[2] * M[6 + j];
        }
        const float ca = V0[0] * V0[0] + V0[1] * V0[1] + V0[2] * V0[2] + 0.3f;
        const float cbv = V0[0] * V1[0] + V0[1] * V1[1] + V0[2] * V1[2];
        const float ccv = V1[0] * V1[0] + V1[1] * V1[1] + V1[2] * V1[2] + 0.3f;
        const float det = ca * ccv - cbv * cbv;
        const float idet = vis ? 1.0f / det : 0.f;
        const float KA = ccv * idet, KB = -cbv * idet, KC = ca * idet;
        int am = 0;
        float smax = v[3];
        if (v[4] > smax) { smax = v[4]; am = 1; }
        if (v[5] > smax) { smax = v[5]; am = 2; }
        const float es = vis ? expf(smax * rz) : 0.f;

        // ---- backward ----
        const float gcol[3] = {up[0], up[1], up[2]}, gw = up[3], go = up[4];
        float dt[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
        float dP[3] = {0.f, 0.f, 0.f}, dY[12];
        // conic -> Sigma_2D:  dSigma = -K Gk K, Gk = [[gA, gB/2], [gB/2, gC]]
        const float G00 = up[7], G01 = 0.5f * up[8], G11 = up[9];
        const float KG00 = KA * G00 + KB * G01, KG01 = KA * G01 + KB * G11;
        const float KG10 = KB * G00 + KC * G01, KG11 = KB * G01 + KC * G11;
        const float dS00 = -(KG00 * KA + KG01 * KB), dS01 = -(KG00 * KB + KG01 * KC);
        const float dS11 = -(KG10 * KB + KG11 * KC);
        const float ga = dS00, gb = 2.0f * dS01, gc = dS11;
        float dV0[3], dV1[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dV0[j] = 2.0f * ga * V0[j] + gb * V1[j];
            dV1[j] = gb * V0[j] + 2.0f * gc * V1[j];
        }
        float dT0[3], dT1[3], dR[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            dT0[k] = dV0[0] * M[3 * k] + dV0[1] * M[3 * k + 1] + dV0[2] * M[3 * k + 2];
            dT1[k] = dV1[0] * M[3 * k] + dV1[1] * M[3 * k + 1] + dV1[2] * M[3 * k + 2];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float dM = T0[k] * dV0[j] + T1[k] * dV1[j];
                dR[3 * k + j] = dM * v[3 + j];
                ds[j] += dM * R[3 * k + j];
            }
        }
        const float dJ00 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
        const float dJ02 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
        const float dJ11 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
        const float dJ12 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
        const float rz2 = rz * rz;
        dt[2] += -dJ00 * cam.fx * rz2 - dJ11 * cam.fy * rz2;
        if (!cx_) {
            dt[0] += -dJ02 * cam.fx * rz2;
            dt[2] += dJ02 * 2.0f * cam.fx * t[0] * rz2 * rz;
        } else {
            dt[2] += dJ02 * cam.fx * uc * rz2;
        }
        if (!cy_) {
            dt[1] += -dJ12 * cam.fy * rz2;
            dt[2] += dJ12 * 2.0f * cam.fy * t[1] * rz2 * rz;
        } else {
            dt[2] += dJ12 * cam.fy * vc * rz2;
        }
        // pixel mean
        dt[0] += up[5] * cam.fx * rz;
        dt[1] += up[6] * cam.fy * rz;
        dt[2] += -(up[5] * cam.fx * t[0] + up[6] * cam.fy * t[1]) * rz2;
        // Eq. 3
        const float dphi = gw * (2.0f * phi + rz2);
        dt[2] += gw * (-2.0f * phi * rz2 * rz - es * smax * rz2);
        ds[am] += gw * es * rz;
        // colour
        float dbase[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            dbase[ch] = cbase[ch] > 0.0f ? gcol[ch] : 0.0f;
            dY[ch] = C0 * dbase[ch];
            dY[3 + ch] = -C1 * P[1] * dbase[ch];
            dY[6 + ch] = C1 * P[2] * dbase[ch];
            dY[9 + ch] = -C1 * P[0] * dbase[ch];
            dP[0] += -C1 * v[20 + ch] * dbase[ch];
            dP[1] += -C1 * v[14 + ch] * dbase[ch];
            dP[2] += C1 * v[17 + ch] * dbase[ch];
        }
        float d_o_stored = 0.0f;
        float dqh[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (kMLP) {
            // Eq. 4 head: phi = ReLU(y0), o = sigmoid(y1), residual y2..4
            float d3[5];
            d3[0] = yv[0] > 0.0f ? dphi : 0.0f;
            d3[1] = go * o * (1.0f - o);
            d3[2] = kResidual ? dbase[0] : 0.0f;
            d3[3] = kResidual ? dbase[1] : 0.0f;
            d3[4] = kResidual ? dbase[2] : 0.0f;
            if (!vis) d3[0] = d3[1] = d3[2] = d3[3] = d3[4] = 0.0f;
            const int row = warp * 32 + lane;
#pragma unroll
            for (int k = 0; k < 8; ++k) sm.d3[row * kD3S + k] = k < kMlpOut ? d3[k] : 0.0f;
#pragma unroll
            for (int k = 0; k < kMlpOut; ++k) sb3[k] += d3[k];
            __syncwarp();
            mlp_d2_warp(sm, warp, lane);
            __syncthreads();
            mlp_wgrad2_cta(sm, warp, lane, wacc);
            __syncthreads();
            mlp_d1_warp(sm, warp, lane);
            __syncthreads();
            mlp_wgrad1_cta(sm, warp, lane, wacc);
            float dx[kDxS];
#pragma unroll
            for (int k = 0; k < kDxS; k += 4) {
                const float4 q4 = *reinterpret_cast<const float4 *>(&sm.dx[row * kDxS + k]);
                dx[k] = q4.x;
                dx[k + 1] = q4.y;
                dx[k + 2] = q4.z;
                dx[k + 3] = q4.w;
            }
            dP[0] += dx[0];
            dP[1] += dx[1];
            dP[2] += dx[2];
            ds[0] += dx[3];
            ds[1] += dx[4];
            ds[2] += dx[5];
            dqh[0] += dx[6];
            dqh[1] += dx[7];
            dqh[2] += dx[8];
            dqh[3] += dx[9];
#pragma unroll
            for (int k = 0; k < 12; ++k) dY[k] += dx[10 + k];
        } else {
            d_o_stored = go;
            (void)dphi;
        }
        if (!valid) continue;
        float *out = d_attrs + (size_t)(args.perm ? args.perm[i] : (uint32_t)i) * kRec;
        if (!vis) {
#pragma unroll
            for (int k = 0; k < kRec; ++k) out[k] = 0.f;
            continue;
        }
        // R(q_hat) -> q_hat
        const float w_ = qw, x_ = qx, y_ = qy, z_ = qz;
        dqh[0] += 2.f * (-z_ * dR[1] + y_ * dR[2] + z_ * dR[3] - x_ * dR[5] - y_ * dR[6] + x_ * dR[7]);
        dqh[1] += 2.f * (y_ * dR[1] + z_ * dR[2] + y_ * dR[3] - 2.f * x_ * dR[4] - w_ * dR[5] +
                         z_ * dR[6] + w_ * dR[7] - 2.f * x_ * dR[8]);
        dqh[2] += 2.f * (-2.f * y_ * dR[0] + x_ * dR[1] + w_ * dR[2] + x_ * dR[3] + z_ * dR[5] -
                         w_ * dR[6] + z_ * dR[7] - 2.f * y_ * dR[8]);
        dqh[3] += 2.f * (-2.f * z_ * dR[0] - w_ * dR[1] + x_ * dR[2] + w_ * dR[3] - 2.f * z_ * dR[4] +
                         y_ * dR[5] + x_ * dR[6] + y_ * dR[7]);
        const float qd = qw * dqh[0] + qx * dqh[1] + qy * dqh[2] + qz * dqh[3];
        dq[0] = (dqh[0] - qw * qd) * iqn;
        dq[1] = (dqh[1] - qx * qd) * iqn;
        dq[2] = (dqh[2] - qy * qd) * iqn;
        dq[3] = (dqh[3] - qz * qd) * iqn;
        // t = W mu + t_cam, P = (mu - c) / |mu - c|
        const float pd = P[0] * dP[0] + P[1] * dP[1] + P[2] * dP[2];
        float dmu[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            dmu[j] = W[j] * dt[0] + W[3 + j] * dt[1] + W[6 + j] * dt[2] + (dP[j] - P[j] * pd) * idn;
        out[0] = dmu[0];
        out[1] = dmu[1];
        out[2] = dmu[2];
        out[3] = ds[0];
        out[4] = ds[1];
        out[5] = ds[2];
        out[6] = dq[0];
        out[7] = dq[1];
        out[8] = dq[2];
        out[9] = dq[3];
        out[10] = d_o_stored;
#pragma unroll
        for (int k = 0; k < 12; ++k) out[11 + k] = dY[k];
        out[23] = 0.f;
    }
    if constexpr (kMLP) {
        // every element of this CTA's partial row is owned by one (lane, register)
        float *P = partials + (size_t)blockIdx.x * kMlpGrad;
        const int g = lane >> 2, t = lane & 3;
        const int m0 = warp * 16 + g, m1 = m0 + 8;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            P[kOffW2 + m0 * kMlpHidden + c] = wacc.w2[nt][0];
            P[kOffW2 + m0 * kMlpHidden + c + 1] = wacc.w2[nt][1];
            P[kOffW2 + m1 * kMlpHidden + c] = wacc.w2[nt][2];
            P[kOffW2 + m1 * kMlpHidden + c + 1] = wacc.w2[nt][3];
        }
        if (t == 0) {
            P[kOffB2 + m0] = wacc.w2[8][0];
            P[kOffB2 + m1] = wacc.w2[8][2];
        }
#pragma unroll
        for (int ft = 0; ft < 3; ++ft) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = ft * 8 + 2 * t + h;
                if (f < kMlpIn) {
                    P[kOffW1 + m0 * kMlpIn + f] = wacc.w1[ft][h];
                    P[kOffW1 + m1 * kMlpIn + f] = wacc.w1[ft][2 + h];
                } else if (f == kXOnesCol) {
                    P[kOffB1 + m0] = wacc.w1[ft][h];
                    P[kOffB1 + m1] = wacc.w1[ft][2 + h];
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * t + h;
            if (k < kMlpOut) {
                P[kOffW3 + k * kMlpHidden + m0] = wacc.w3[h];
                P[kOffW3 + k * kMlpHidden + m1] = wacc.w3[2 + h];
            }
        }
#pragma unroll
        for (int k = 0; k < kMlpOut; ++k) {
            float x = sb3[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) sm.b3[warp][k] = x;
        }
        __syncthreads();
        if (threadIdx.x < kMlpOut) {
            float x = 0.f;
            for (int w = 0; w < kMlpThreads / 32; ++w) x += sm.b3[w][threadIdx.x];
            P[kOffB3 + threadIdx.x] = x;
        }
    }
}

__global__ void k_mlp_grad_reduce(const float *__restrict__ partials, int nparts,
                                  float *__restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpGrad) return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += partials[(size_t)c * kMlpGrad + e];
    out[e] = s;
}

template <bool kFP16, bool kMLP, bool kRes>
cudaError_t launch_pre_bwd(const RenderArgs &a, int blocks, const float *gG, float *d_attrs,
                           float *partials, cudaStream_t stream) {
    const size_t smem = kMLP ? sizeof(BwdSmem) : 16;
    auto kern = k_preprocess_bwd<kFP16, kMLP, kRes>;
    if (kMLP) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<blocks, kMlpThreads, smem, stream>>>(a, gG, d_attrs, partials);
    return cudaGetLastError();
}

}  // namespace

int mlp_grad_size() { return kMlpGrad; }
int grad_record_size() { return kGRec; }
int pre_bwd_blocks(int64_t n, int sm_count) {
    int64_t b = (n + kMlpThreads - 1) / kMlpThreads;
    const int64_t cap = 2 * (int64_t)sm_count;
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

cudaError_t launch_backward(const RenderArgs &a, int sm_count, const float *dL_drgb,
                            const float *aux, float *gG, float *d_attrs, float *d_mlp,
                            float *partials, cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    cudaError_t e = cudaMemsetAsync(gG, 0, (size_t)a.n * kGRec * sizeof(float), stream);
    if (e != cudaSuccess) return e;
    k_raster_bwd<<<T, kBwdThreads, 0, stream>>>(a, dL_drgb, aux, gG);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int blocks = pre_bwd_blocks(a.n, sm_count);
    const bool fp16 = a.precision == MGS_PREC_FP16;
    if (a.use_mlp) {
        if (a.rgb_residual)
            e = fp16 ? launch_pre_bwd<true, true, true>(a, blocks, gG, d_attrs, partials, stream)
                     : launch_pre_bwd<false, true, true>(a, blocks, gG, d_attrs, partials, stream);
        else
            e = fp16 ? launch_pre_bwd<true, true, false>(a, blocks, gG, d_attrs, partials, stream)
                     : launch_pre_bwd<false, true, false>(a, blocks, gG, d_attrs, partials, stream);
        if (e != cudaSuccess) return e;
        if (d_mlp) {
            k_mlp_grad_reduce<<<(kMlpGrad + 255) / 256, 256, 0, stream>>>(partials, blocks, d_mlp);
            e = cudaGetLastError();
        }
        return e;
    }
    e = fp16 ? launch_pre_bwd<true, false, false>(a, blocks, gG, d_attrs, partials, stream)
             : launch_pre_bwd<false, false, false>(a, blocks, gG, d_attrs, partials, stream);
    if (e == cudaSuccess && d_mlp)
        e = cudaMemsetAsync(d_mlp, 0, (size_t)kMlpGrad * sizeof(float), stream);
    return e;
}

}  // namespace mgs
