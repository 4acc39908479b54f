// Per-pixel depth-aware, order-independent accumulation (Sec. 3.1, Eq. 2):
//
//   A = sum_i c_i a_i w_i,  B = sum_i a_i w_i,  T = prod_i (1 - a_i)
//   C = (1 - T) A / B + T c_bg          (foreground term 0 when B = 0)
//
// One CTA per 16x16 tile, 128 threads, each thread owning two horizontally
// adjacent pixels (packed FP32x2 arithmetic).  Each warp owns an 8x8 block and
// walks the tile's Gaussian list itself, testing each entry against its block
// with a conservative bound and compacting (ballot) the candidates before
// accumulating them in registers.  No atomics, no sort: every pixel is owned
// by exactly one thread.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;

typedef unsigned long long f2;  // two packed FP32 lanes

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Staged Gaussian: five 16-byte words of duplicated pairs, so every operand
// of the packed arithmetic comes straight from one shared-memory load.
//   s0 = {m_x, m_x, m_y, m_y}      s1 = {l11, l11, l21, l21}
//   s2 = {l22, l22, log2 o, log2 o} s3 = {-w, -w, -w c_r, -w c_r}
//   s4 = {-w c_g, -w c_g, -w c_b, -w c_b}

// Can Gaussian (m, l) include any pixel centre of the block centred at (bx, by)
// with half extents (hx, hy)?  Sound for the exact FP32 test: the slab bounds
// |e1| <= 3 and |e2| <= 3 hold for every included pixel, and the margin
// (2^-18 relative) covers the rounding of both evaluations.
__device__ __forceinline__ bool block_may_hit(float mx, float my, float l11, float l21, float l22,
                                              float bx, float by, float hx, float hy) {
    const float dxb = bx - mx, dyb = by - my;
    const float e1c = fabsf(fmaf(l11, dxb, l21 * dyb));
    const float h1 = fmaf(fabsf(l11), hx, fabsf(l21) * hy);
    const float m1 = 3.814697265625e-06f *
                     (fabsf(l11) * (fabsf(dxb) + hx) + fabsf(l21) * (fabsf(dyb) + hy) + 4.0f);
    const float e2c = fabsf(l22 * dyb);
    const float h2 = fabsf(l22) * hy;
    const float m2 = 3.814697265625e-06f * (fabsf(l22) * (fabsf(dyb) + hy) + 4.0f);
    return (e1c - h1 <= 3.0f + m1) && (e2c - h2 <= 3.0f + m2);
}

// One CTA per tile; warp w owns the 8x8 pixel block (w & 1, w >> 1) of the
// tile, lane l the pixel pair (2 (l & 3), l >> 2) of that block.  Each warp
// streams the tile's list on its own (no block-wide barrier): 32 entries at a
// time, one per lane, are fetched, tested against the warp's block, and the
// candidates are compacted into the warp's shared-memory buffer and then
// accumulated by all lanes.
template <bool kAux, bool kCount>
__global__ void __launch_bounds__(kThreads) k_raster(RenderArgs args) {
    __shared__ ulonglong2 buf[kWarps][5][32];
    const DevCamera &cam = args.cam;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile + 8 * (warp & 1), by0 = ty * kTile + 8 * (warp >> 1);
    const int px = bx0 + 2 * (lane & 3);
    const int py = by0 + (lane >> 2);

    if (args.status->last_pairs > args.capacity) return;  // overflowed: lists incomplete

    const uint32_t start = args.tile_offsets[tile];
    const uint32_t end = args.tile_offsets[tile + 1];
    const bool no_cull = (args.flags & MGS_FLAG_NO_CULL) != 0;
    const float bx = (float)bx0 + 4.0f, by = (float)by0 + 4.0f;

    const f2 pxc = pk((float)px + 0.5f, (float)px + 1.5f);
    const f2 pyc = pk((float)py + 0.5f, (float)py + 0.5f);
    const float kq = -0.72134752044448170f;  // -log2(e) / 2
    const f2 kq2 = pk(kq, kq);
    f2 Ar = 0ull, Ag = 0ull, Ab = 0ull, B = 0ull;
    f2 T = pk(1.0f, 1.0f);
    int cnt0 = 0, cnt1 = 0;
    ulonglong2(*wb)[32] = buf[warp];

    for (uint32_t base = start; base < end; base += 32) {
        const uint32_t j = base + lane;
        bool cand = false;
        float4 a, b, c;
        if (j < end) {
            const uint32_t gid = __ldg(&args.gids[j]);
            a = __ldg(&args.rec[gid].a);
            b = __ldg(&args.rec[gid].b);
            c = __ldg(&args.rec[gid].c);
            cand = no_cull || block_may_hit(a.x, a.y, a.z, a.w, b.x, bx, by, 3.5f, 3.5f);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (cand) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            wb[0][pos] = make_ulonglong2(pk(a.x, a.x), pk(a.y, a.y));
            wb[1][pos] = make_ulonglong2(pk(a.z, a.z), pk(a.w, a.w));
            wb[2][pos] = make_ulonglong2(pk(b.x, b.x), pk(b.y, b.y));
            wb[3][pos] = make_ulonglong2(pk(b.z, b.z), pk(b.w, b.w));
            wb[4][pos] = make_ulonglong2(pk(c.x, c.x), pk(c.y, c.y));
        }
        __syncwarp();
        const int n = __popc(bal);
#pragma unroll 2
        for (int k = 0; k < n; ++k) {
            const ulonglong2 s0 = wb[0][k], s1 = wb[1][k], s2 = wb[2][k];
            // inclusion test (exact FP32 sequence)
            const f2 dx = sub2(pxc, s0.x);
            const f2 dy = sub2(pyc, s0.y);
            const f2 e1 = fma2(s1.x, dx, mul2(s1.y, dy));
            const f2 e2 = mul2(s2.x, dy);
            const f2 q = fma2(e1, e1, mul2(e2, e2));
            // a = min(0.99, o 2^(-q log2(e) / 2)), kept negated
            const f2 arg = fma2(q, kq2, s2.y);
            float q0, q1, g0, g1;
            upk(q, q0, q1);
            upk(arg, g0, g1);
            float n0 = fmaxf(-ex2(g0), -0.99f);
            float n1 = fmaxf(-ex2(g1), -0.99f);
            n0 = q0 <= 9.0f ? n0 : 0.0f;
            n1 = q1 <= 9.0f ? n1 : 0.0f;
            if (kCount) {
                cnt0 += q0 <= 9.0f;
                cnt1 += q1 <= 9.0f;
            }
            const f2 na = pk(n0, n1);
            const ulonglong2 s3 = wb[3][k], s4 = wb[4][k];
            Ar = fma2(na, s3.y, Ar);
            Ag = fma2(na, s4.x, Ag);
            Ab = fma2(na, s4.y, Ab);
            B = fma2(na, s3.x, B);
            T = fma2(na, T, T);
        }
        __syncwarp();
    }

    if (py >= cam.height) return;
    float ar[2], ag[2], ab[2], bb[2], tt[2];
    upk(Ar, ar[0], ar[1]);
    upk(Ag, ag[0], ag[1]);
    upk(Ab, ab[0], ab[1]);
    upk(B, bb[0], bb[1]);
    upk(T, tt[0], tt[1]);
    const int cnts[2] = {cnt0, cnt1};
    const int64_t HW = (int64_t)cam.width * cam.height;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int x = px + k;
        if (x >= cam.width) break;
        const int64_t p = (int64_t)py * cam.width + x;
        const float fg = bb[k] > 0.0f ? (1.0f - tt[k]) / bb[k] : 0.0f;
        float *o = args.out_rgb + 3 * p;
        o[0] = fmaf(fg, ar[k], tt[k] * args.bg[0]);
        o[1] = fmaf(fg, ag[k], tt[k] * args.bg[1]);
        o[2] = fmaf(fg, ab[k], tt[k] * args.bg[2]);
        if (kAux) {
            args.out_aux[p] = ar[k];
            args.out_aux[HW + p] = ag[k];
            args.out_aux[2 * HW + p] = ab[k];
            args.out_aux[3 * HW + p] = bb[k];
            args.out_aux[4 * HW + p] = tt[k];
        }
        if (kCount) args.out_count[p] = cnts[k];
    }
}

template <bool kAux, bool kCount>
cudaError_t launch_t(const RenderArgs &a, cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    k_raster<kAux, kCount><<<T, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster(const RenderArgs &a, cudaStream_t stream) {
    const bool aux = a.out_aux != nullptr, cnt = a.out_count != nullptr;
    if (aux && cnt) return launch_t<true, true>(a, stream);
    if (aux) return launch_t<true, false>(a, stream);
    if (cnt) return launch_t<false, true>(a, stream);
    return launch_t<false, false>(a, stream);
}

}  // namespace mgs
