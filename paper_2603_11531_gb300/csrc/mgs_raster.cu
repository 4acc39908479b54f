// Per-pixel depth-aware, order-independent accumulation (Sec. 3.1, Eq. 2):
//
//   A = sum_i c_i a_i w_i,  B = sum_i a_i w_i,  T = prod_i (1 - a_i)
//   C = (1 - T) A / B + T c_bg          (foreground term 0 when B = 0)
//
// FP32 scenes (k_raster): one CTA per 16x16 tile, 64 threads, each thread
// owning four horizontally adjacent pixels (two packed FP32x2 pairs).  Each
// warp owns a 16x8 block and walks the tile's Gaussian list itself, testing
// each entry against its block with a conservative bound (block_may_hit) and
// compacting (ballot) the candidates before accumulating them in registers.
//
// FP16-attribute scenes (k_raster_tc): four warps of 8x8 pixels per tile;
// alpha is still computed, tested and multiplied into T in FP32 exactly as
// above, but a_i w_i c_i and a_i w_i are summed on the tensor cores by
// mma.sync (m16n8k8, FP16 operands, FP32 accumulation) with the weights split
// into FP16 high and low parts, which leaves alpha's FP16 rounding (relative
// 2^-12 per term) as the only extra error; tiles listing a Gaussian outside
// the FP16 weight range take the FP32 code.
//
// No atomics, no sort: every pixel is owned by exactly one thread, and a
// tile's list is accumulated in whatever order binning stored it.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kThreads = 64;
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

// Accumulates one staged Gaussian into a thread's four pixels (two pairs).
template <bool kCount, bool kDepth>
__device__ __forceinline__ void accumulate(const ulonglong2 (*wb)[32], int k, f2 pxa, f2 pxb,
                                           f2 pyc, f2 kq2, f2 (&A)[2][3], f2 (&B)[2],
                                           f2 (&T)[2], f2 (&AD)[2], int (&cnt)[4]) {
    const ulonglong2 s0 = wb[0][k], s1 = wb[1][k], s2 = wb[2][k];
    // inclusion test (exact FP32 sequence); the row terms are shared by both pairs
    const f2 dy = sub2(pyc, s0.y);
    const f2 ldy = mul2(s1.y, dy);
    const f2 e2 = mul2(s2.x, dy);
    const f2 e2s = mul2(e2, e2);
    const f2 dxa = sub2(pxa, s0.x);
    const f2 dxb = sub2(pxb, s0.x);
    const f2 e1a = fma2(s1.x, dxa, ldy);
    const f2 e1b = fma2(s1.x, dxb, ldy);
    const f2 qa = fma2(e1a, e1a, e2s);
    const f2 qb = fma2(e1b, e1b, e2s);
    // a = min(0.99, o 2^(-q log2(e) / 2)), kept negated
    const f2 ga = fma2(qa, kq2, s2.y);
    const f2 gb = fma2(qb, kq2, s2.y);
    float q[4], g[4], n[4];
    upk(qa, q[0], q[1]);
    upk(qb, q[2], q[3]);
    upk(ga, g[0], g[1]);
    upk(gb, g[2], g[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        n[i] = q[i] <= 9.0f ? fmaxf(-ex2(g[i]), -0.99f) : 0.0f;
        if (kCount) cnt[i] += q[i] <= 9.0f;
    }
    const ulonglong2 s3 = wb[3][k], s4 = wb[4][k];
    const f2 na[2] = {pk(n[0], n[1]), pk(n[2], n[3])};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        A[h][0] = fma2(na[h], s3.y, A[h][0]);
        A[h][1] = fma2(na[h], s4.x, A[h][1]);
        A[h][2] = fma2(na[h], s4.y, A[h][2]);
        B[h] = fma2(na[h], s3.x, B[h]);
        T[h] = fma2(na[h], T[h], T[h]);
    }
    if (kDepth) {
        const ulonglong2 s5 = wb[5][k];   // {-w d, -w d, 0, 0}
        AD[0] = fma2(na[0], s5.x, AD[0]);
        AD[1] = fma2(na[1], s5.x, AD[1]);
    }
}

// Rasterises one tile with one CTA (two warps); warp w owns the 16x8 pixel
// block of rows 8w..8w+7, lane l the four pixels (4 (l & 3) .. +3, l >> 2) of
// that block.  Each warp streams the tile's list on its own (no block-wide
// barrier): 32 entries at a time, one per lane (the next 32 are fetched while
// the current ones are accumulated), are tested against the warp's block,
// compacted into the warp's shared-memory buffer (ballot) and accumulated by
// all lanes.
template <bool kAux, bool kCount, bool kDepth = false>
__device__ __forceinline__ void raster_tile(const RenderArgs &args, int tile,
                                            ulonglong2 (*buf)[kDepth ? 6 : 5][32]) {
    const DevCamera &cam = args.cam;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile, by0 = ty * kTile + 8 * warp;
    const int px = bx0 + 4 * (lane & 3);
    const int py = by0 + (lane >> 2);

    const uint32_t start = args.tile_offsets[tile];
    const uint32_t end = args.tile_offsets[tile + 1];
    const bool no_cull = (args.flags & MGS_FLAG_NO_CULL) != 0;
    const float bx = (float)bx0 + 8.0f, by = (float)by0 + 4.0f;

    const f2 pxa = pk((float)px + 0.5f, (float)px + 1.5f);
    const f2 pxb = pk((float)px + 2.5f, (float)px + 3.5f);
    const f2 pyc = pk((float)py + 0.5f, (float)py + 0.5f);
    const float kq = -0.72134752044448170f;  // -log2(e) / 2
    const f2 kq2 = pk(kq, kq);
    f2 A[2][3] = {{0ull, 0ull, 0ull}, {0ull, 0ull, 0ull}};
    f2 B[2] = {0ull, 0ull};
    f2 T[2] = {pk(1.0f, 1.0f), pk(1.0f, 1.0f)};
    f2 AD[2] = {0ull, 0ull};
    int cnt[4] = {0, 0, 0, 0};
    ulonglong2(*wb)[32] = buf[warp];

    // list entries two batches ahead, their records one batch ahead (the
    // dependent record loads never wait on the list load)
    float4 a_n = make_float4(0.f, 0.f, 0.f, 0.f), b_n = a_n, c_n = a_n;
    uint32_t gid_nn = 0;
    if (start + lane < end) {
        const uint32_t gid = __ldg(&args.gids[start + lane]);
        a_n = __ldg(&args.rec[gid].a);
        b_n = __ldg(&args.rec[gid].b);
        c_n = __ldg(&args.rec[gid].c);
    }
    if (start + 32 + lane < end) gid_nn = __ldg(&args.gids[start + 32 + lane]);
    for (uint32_t base = start; base < end; base += 32) {
        const uint32_t j = base + lane;
        const float4 a = a_n, b = b_n, c = c_n;
        const bool cand =
            j < end && (no_cull || block_may_hit(a.x, a.y, a.z, a.w, b.x, bx, by, 7.5f, 3.5f));
        if (j + 32 < end) {
            const uint32_t gid = gid_nn;
            a_n = __ldg(&args.rec[gid].a);
            b_n = __ldg(&args.rec[gid].b);
            c_n = __ldg(&args.rec[gid].c);
        }
        if (j + 64 < end) gid_nn = __ldg(&args.gids[j + 64]);
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (cand) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            wb[0][pos] = make_ulonglong2(pk(a.x, a.x), pk(a.y, a.y));
            wb[1][pos] = make_ulonglong2(pk(a.z, a.z), pk(a.w, a.w));
            wb[2][pos] = make_ulonglong2(pk(b.x, b.x), pk(b.y, b.y));
            wb[3][pos] = make_ulonglong2(pk(b.z, b.z), pk(b.w, b.w));
            wb[4][pos] = make_ulonglong2(pk(c.x, c.x), pk(c.y, c.y));
            if (kDepth) wb[5][pos] = make_ulonglong2(pk(c.w, c.w), 0ull);   // -w d
        }
        __syncwarp();
        const int nc = __popc(bal);
#pragma unroll 2
        for (int k = 0; k < nc; ++k)
            accumulate<kCount, kDepth>(wb, k, pxa, pxb, pyc, kq2, A, B, T, AD, cnt);
        __syncwarp();
    }

    if (py >= cam.height) return;
    float ar[4], ag[4], ab[4], bb[4], tt[4], ad[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        upk(AD[h], ad[2 * h], ad[2 * h + 1]);
        upk(A[h][0], ar[2 * h], ar[2 * h + 1]);
        upk(A[h][1], ag[2 * h], ag[2 * h + 1]);
        upk(A[h][2], ab[2 * h], ab[2 * h + 1]);
        upk(B[h], bb[2 * h], bb[2 * h + 1]);
        upk(T[h], tt[2 * h], tt[2 * h + 1]);
    }
    const int64_t HW = (int64_t)cam.width * cam.height;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
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
        if (kCount) args.out_count[p] = cnt[k];
        if (kDepth) args.out_depth[p] = bb[k] > 0.0f ? ad[k] / bb[k] : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Tensor-core accumulation of A and B (FP16-attribute scenes).
//
// One CTA (four warps) per tile; warp w owns the 8x8 block at
// (8 (w % 2), 8 (w / 2)) of the tile.  A warp's 64 pixels are the M = 64 rows
// of four m16n8k8 tiles: lane (g, t) = (lane / 4, lane % 4) owns the eight
// pixels x = 0..7 of the block's row g (rows g and g + 8 of m-tile i are
// pixels 2i and 2i + 1), shared by the four lanes of its quad.  Candidates
// are gathered into chunks of 8 Gaussians (the K dimension); lane t of a
// quad evaluates chunk entries 2t and 2t + 1 at its pixels -- one packed
// FP32x2 operation serves both, and the packed pair of alphas is exactly the
// A fragment the lane holds.  B = the chunk's weights [w c_r, w c_g, w c_b, w]
// as FP16 high parts (columns 0-3) and low parts (columns 4-7), so column c +
// column c + 4 is the sum with a 22-bit weight; preprocessing writes these
// FP16 weights once per Gaussian, and binning rescales them by a power of two
// when the frame's largest weight would overflow FP16 (the scale cancels in
// A / B and is divided out here).  T stays in FP32 FMAs.  Tiles listing a Gaussian
// outside that scale's range (kTileWide) are rasterised by the FMA tile code.
constexpr int kTcThreads = 128;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kChunk = 8;        // candidates per MMA (K)
constexpr int kRing = 64;        // candidate slots per warp: eight chunks (a power of two)

// Ring slot s stores its geometry in pair-interleaved words, so that lane t
// reads the two entries 2t, 2t + 1 of a chunk with one 16-byte load each:
//   geo[0][s / 2] = {m_x(a), m_x(b), m_y(a), m_y(b)}
//   geo[1][s / 2] = {l11(a), l11(b), l21(a), l21(b)}
//   geo[2][s / 2] = {l22(a), l22(b), log2 o(a), log2 o(b)}   (a = even slot)
struct TcSmem {
    float4 geo[kTcWarps][3][kRing / 2];
    uint4 wt[kTcWarps][kRing];            // slot s: its 8 FP16 weight columns
    float2 wd[kTcWarps][kRing / 2];       // depth image only: w d of slots 2p, 2p + 1
};

__device__ __forceinline__ uint32_t h2bits(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// One chunk of 8 candidates starting at ring slot c0 (a multiple of 8): the
// lane's entries 2t, 2t + 1 at its eight pixels (same FP32 sequence as
// accumulate()), T updated, alphas packed to FP16 and summed by four MMAs.
// kDepth: also AD[j] += (a, b) * (w d of the two entries), the FP32 numerator
// of the depth image (Eq. 5), kept as two partial sums per pixel.
template <bool kCount, bool kClamp, bool kDepth = false>
__device__ __forceinline__ void tc_chunk(const float4 (*geo)[kRing / 2], const uint4 *wt,
                                         int c0, int g, int t, const f2 (&pxc)[8], f2 pyc,
                                         f2 kq2, float (&T)[8], float (&D)[4][4], int (&cnt)[8],
                                         const float2 *wd = nullptr, f2 *AD = nullptr) {
    const int pr = (c0 >> 1) + t;
    f2 wdp = 0ull;
    if constexpr (kDepth) wdp = pk(wd[pr].x, wd[pr].y);
    const float4 q0 = geo[0][pr], q1 = geo[1][pr], q2 = geo[2][pr];
    const f2 mx = pk(q0.x, q0.y), my = pk(q0.z, q0.w);
    const f2 l11 = pk(q1.x, q1.y), l21 = pk(q1.z, q1.w);
    const f2 l22 = pk(q2.x, q2.y), lo = pk(q2.z, q2.w);
    const f2 dy = sub2(pyc, my);
    const f2 ldy = mul2(l21, dy);
    const f2 e2 = mul2(l22, dy);
    const f2 e2s = mul2(e2, e2);
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const f2 dx = sub2(pxc[j], mx);
        const f2 e1 = fma2(l11, dx, ldy);
        const f2 q = fma2(e1, e1, e2s);
        const f2 gg = fma2(q, kq2, lo);
        float qa, qb, ga, gb;
        upk(q, qa, qb);
        upk(gg, ga, gb);
        float aa = ex2(ga), ab = ex2(gb);
        if (kClamp) {
            aa = fminf(aa, 0.99f);
            ab = fminf(ab, 0.99f);
        }
        aa = qa <= 9.0f ? aa : 0.0f;
        ab = qb <= 9.0f ? ab : 0.0f;
        if (kCount) cnt[j] += (qa <= 9.0f) + (qb <= 9.0f);
        T[j] = fmaf(-aa, T[j], T[j]);
        T[j] = fmaf(-ab, T[j], T[j]);
        if constexpr (kDepth) AD[j] = fma2(pk(aa, ab), wdp, AD[j]);
        a[j] = h2bits(aa, ab);            // k = 2t (low half), 2t + 1
    }
    const unsigned short *wa = reinterpret_cast<const unsigned short *>(wt + c0 + 2 * t);
    const uint32_t b0 = (uint32_t)wa[g] | ((uint32_t)wa[8 + g] << 16);   // column g, k = 2t, 2t + 1
#pragma unroll
    for (int i = 0; i < 4; ++i) mma_k8(D[i], a[2 * i], a[2 * i + 1], b0);   // pixels 2i, 2i + 1
}

template <bool kAux, bool kCount, bool kDepth = false>
__device__ __forceinline__ void raster_tile_tc(const RenderArgs &args, int tile, TcSmem &sm) {
    const DevCamera &cam = args.cam;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int bx0 = tx * kTile + 8 * (warp & 1), by0 = ty * kTile + 8 * (warp >> 1);
    const int xb = bx0;
    const int py = by0 + g;
    float4(*geo)[kRing / 2] = sm.geo[warp];
    uint4 *wt = sm.wt[warp];
    float2 *wd = sm.wd[warp];

    const uint32_t start = args.tile_offsets[tile];
    const uint32_t end = args.tile_offsets[tile + 1];
    const bool no_cull = (args.flags & MGS_FLAG_NO_CULL) != 0;
    const float bcx = (float)bx0 + 4.0f, bcy = (float)by0 + 4.0f;
    // weight scale 2^(14 - e) when the frame's largest weight has exponent e >= 14
    const int we = (int)((args.status->wmax_frame_bits >> 23) & 0xFFu) - 127;
    const float wscale = we >= 14 ? __int_as_float((127 + 14 - we) << 23) : 1.0f;
    const float kLogClamp = -0.014499569695115089f;   // log2(0.99)

    f2 pxc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) pxc[j] = pk((float)(xb + j) + 0.5f, (float)(xb + j) + 0.5f);
    const f2 pyc = pk((float)py + 0.5f, (float)py + 0.5f);
    const float kq = -0.72134752044448170f;  // -log2(e) / 2
    const f2 kq2 = pk(kq, kq);
    float T[8];
    float D[4][4];
    int cnt[8];
    f2 AD[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        T[j] = 1.0f;
        cnt[j] = 0;
        AD[j] = 0ull;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) D[i][0] = D[i][1] = D[i][2] = D[i][3] = 0.0f;

    int head = 0, count = 0;          // unprocessed candidates: ring slots [head, head + count)
    uint64_t clamp_mask = 0;          // ring slots whose opacity exceeds 0.99
    // prefetch of the next batch: everything the block test and staging need
    float4 a_n = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 b_n = make_float2(0.f, 0.f);
    uint4 w_n = make_uint4(0u, 0u, 0u, 0u);
    float d_n = 0.f;                      // depth image: -w d
    // list entries are fetched two batches ahead and their records one batch
    // ahead, so the dependent record loads never wait on the list load
    uint32_t gid_nn = 0;
    if (start + lane < end) {
        const uint32_t gid = __ldg(&args.gids[start + lane]);
        a_n = __ldg(&args.rec[gid].a);
        b_n = __ldg(reinterpret_cast<const float2 *>(&args.rec[gid].b));
        w_n = __ldg(&args.wt16[gid]);
        if constexpr (kDepth) d_n = __ldg(&args.rec[gid].c.w);
    }
    if (start + 32 + lane < end) gid_nn = __ldg(&args.gids[start + 32 + lane]);
    for (uint32_t base = start; base < end; base += 32) {
        const uint32_t j = base + lane;
        const float4 a = a_n;
        const float2 b = b_n;
        const uint4 wv = w_n;
        const float dv = d_n;
        const bool cand =
            j < end && (no_cull || block_may_hit(a.x, a.y, a.z, a.w, b.x, bcx, bcy, 3.5f, 3.5f));
        if (j + 32 < end) {
            const uint32_t gid = gid_nn;
            a_n = __ldg(&args.rec[gid].a);
            b_n = __ldg(reinterpret_cast<const float2 *>(&args.rec[gid].b));
            w_n = __ldg(&args.wt16[gid]);
            if constexpr (kDepth) d_n = __ldg(&args.rec[gid].c.w);
        }
        if (j + 64 < end) gid_nn = __ldg(&args.gids[j + 64]);
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        bool clamp = false;
        int pos = 0;
        if (cand) {
            pos = (head + count + __popc(bal & ((1u << lane) - 1u))) & (kRing - 1);
            float *q = reinterpret_cast<float *>(&geo[0][pos >> 1]);
            const int o = pos & 1;
            q[o] = a.x;
            q[2 + o] = a.y;
            q = reinterpret_cast<float *>(&geo[1][pos >> 1]);
            q[o] = a.z;
            q[2 + o] = a.w;
            q = reinterpret_cast<float *>(&geo[2][pos >> 1]);
            q[o] = b.x;
            q[2 + o] = b.y;
            clamp = b.y > kLogClamp;
            wt[pos] = wv;                        // FP16 weights written by preprocessing
            if constexpr (kDepth) reinterpret_cast<float *>(&wd[pos >> 1])[o] = -dv;
        }
        // slots of this batch that need the 0.99 clamp
        const unsigned cb = __ballot_sync(0xffffffffu, clamp);
        if (cb) {
            for (unsigned m = cb; m; m &= m - 1) {
                const int l = __ffs(m) - 1;
                const int p = __shfl_sync(0xffffffffu, pos, l);
                clamp_mask |= 1ull << p;
            }
        }
        __syncwarp();
        count += __popc(bal);
        while (count >= kChunk) {
            if ((clamp_mask >> head) & 0xFFull)
                tc_chunk<kCount, true, kDepth>(geo, wt, head, g, t, pxc, pyc, kq2, T, D, cnt, wd, AD);
            else
                tc_chunk<kCount, false, kDepth>(geo, wt, head, g, t, pxc, pyc, kq2, T, D, cnt, wd, AD);
            clamp_mask &= ~(0xFFull << head);
            head = (head + kChunk) & (kRing - 1);
            count -= kChunk;
        }
        __syncwarp();
    }
    if (count > 0) {
        // pad the last chunk with entries that include no pixel and weigh 0
        if (lane < kChunk - count) {
            const int pos = (head + count + lane) & (kRing - 1);
            const int o = pos & 1;
            float *q = reinterpret_cast<float *>(&geo[0][pos >> 1]);
            q[o] = 1e30f;
            q[2 + o] = 1e30f;
            q = reinterpret_cast<float *>(&geo[1][pos >> 1]);
            q[o] = 1.0f;
            q[2 + o] = 0.0f;
            q = reinterpret_cast<float *>(&geo[2][pos >> 1]);
            q[o] = 1.0f;
            q[2 + o] = 0.0f;
            wt[pos] = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (kDepth) reinterpret_cast<float *>(&wd[pos >> 1])[o] = 0.0f;
        }
        __syncwarp();
        if ((clamp_mask >> head) & 0xFFull)
            tc_chunk<kCount, true, kDepth>(geo, wt, head, g, t, pxc, pyc, kq2, T, D, cnt, wd, AD);
        else
            tc_chunk<kCount, false, kDepth>(geo, wt, head, g, t, pxc, pyc, kq2, T, D, cnt, wd, AD);
    }

    // Quad reduction: columns c and c + 4 (lanes t, t ^ 2), then swap halves
    // (lanes t, t ^ 1); T and counts multiply / add over the four lanes.
    float v[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[i][k] = D[i][k] + __shfl_xor_sync(0xffffffffu, D[i][k], 2);
    float o[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) o[i][k] = __shfl_xor_sync(0xffffffffu, v[i][k], 1);
    float ad[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if constexpr (kDepth) {
            float x, y;
            upk(AD[k], x, y);
            ad[k] = x + y;
            ad[k] += __shfl_xor_sync(0xffffffffu, ad[k], 1);
            ad[k] += __shfl_xor_sync(0xffffffffu, ad[k], 2);
        }
        T[k] *= __shfl_xor_sync(0xffffffffu, T[k], 1);
        T[k] *= __shfl_xor_sync(0xffffffffu, T[k], 2);
        if (kCount) {
            cnt[k] += __shfl_xor_sync(0xffffffffu, cnt[k], 1);
            cnt[k] += __shfl_xor_sync(0xffffffffu, cnt[k], 2);
        }
    }
    if (py >= cam.height) return;
    const float inv = 1.0f / wscale;
    const int64_t HW = (int64_t)cam.width * cam.height;
    const bool even = (t & 1) == 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i != t) continue;   // lane t writes pixels 2t, 2t + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = xb + 2 * i + h;
            if (x >= cam.width) break;
            // v / o: (A_r, A_g) on even lanes, (A_b, B) on odd lanes; k = 2h, 2h + 1
            const float ar = (even ? v[i][2 * h] : o[i][2 * h]) * inv;
            const float ag = (even ? v[i][2 * h + 1] : o[i][2 * h + 1]) * inv;
            const float ab = (even ? o[i][2 * h] : v[i][2 * h]) * inv;
            const float bb = (even ? o[i][2 * h + 1] : v[i][2 * h + 1]) * inv;
            const float tr = T[2 * i + h];
            const int64_t p = (int64_t)py * cam.width + x;
            const float fg = bb > 0.0f ? (1.0f - tr) / bb : 0.0f;
            float *out = args.out_rgb + 3 * p;
            out[0] = fmaf(fg, ar, tr * args.bg[0]);
            out[1] = fmaf(fg, ag, tr * args.bg[1]);
            out[2] = fmaf(fg, ab, tr * args.bg[2]);
            if (kAux) {
                args.out_aux[p] = ar;
                args.out_aux[HW + p] = ag;
                args.out_aux[2 * HW + p] = ab;
                args.out_aux[3 * HW + p] = bb;
                args.out_aux[4 * HW + p] = tr;
            }
            if (kCount) args.out_count[p] = cnt[2 * i + h];
            // FP32 numerator over the tensor-core B (both unscaled)
            if (kDepth) args.out_depth[p] = bb > 0.0f ? ad[2 * i + h] / bb : 0.0f;
        }
    }
}

// Tensor-core accumulation is used for FP16-attribute scenes unless the
// caller asks for the FP32 FMA sums.
__host__ __device__ __forceinline__ bool use_tc(const RenderArgs &a) { return tc_raster(a); }

// One CTA per tile, longest tile lists first.
template <bool kAux, bool kCount, bool kDepth = false>
__global__ void __launch_bounds__(kThreads) k_raster(RenderArgs args) {
    __shared__ ulonglong2 buf[kWarps][kDepth ? 6 : 5][32];
    if (args.status->last_pairs > args.capacity) return;  // overflowed: lists incomplete
    raster_tile<kAux, kCount, kDepth>(args, (int)(args.tile_order[blockIdx.x] & kTileMask), buf);
}

// Tiles that list a Gaussian whose weight the FP16 sums cannot hold next to
// the others (kTileWide, see kWideWeight) take the FP32 FMA tile code on the
// CTA's first two warps.
template <bool kAux, bool kCount, bool kDepth = false>
__global__ void __launch_bounds__(kTcThreads) k_raster_tc(RenderArgs args) {
    __shared__ union {
        TcSmem tc;
        ulonglong2 buf[kWarps][kDepth ? 6 : 5][32];
    } sm;
    if (args.status->last_pairs > args.capacity) return;  // overflowed: lists incomplete
    const uint32_t ord = args.tile_order[blockIdx.x];
    const int tile = (int)(ord & kTileMask);
    if (ord & kTileWide) {
        if (threadIdx.x < kThreads) raster_tile<kAux, kCount, kDepth>(args, tile, sm.buf);
    } else {
        raster_tile_tc<kAux, kCount, kDepth>(args, tile, sm.tc);
    }
}

// Persistent, batched: the tiles of several views (different scenes and
// resolutions) form one work list; resident CTAs pull (view, tile) items from
// an atomic counter until the list is exhausted.  Items are numbered view by
// view (prefix[v] = first item of view v), each view's tiles longest first.
// A CTA has four warps: FP16 views use all four (tensor-core sums), FP32
// views and wide tiles (kTileWide) the first two (FMA sums).
__global__ void __launch_bounds__(kTcThreads) k_raster_batch(const RenderArgs *__restrict__ views,
                                                             const int *__restrict__ prefix,
                                                             int nviews,
                                                             unsigned *__restrict__ counter) {
    __shared__ union {
        ulonglong2 buf[kWarps][5][32];
        TcSmem tc;
    } sm;
    __shared__ int item_s;
    const int total = prefix[nviews];
    for (;;) {
        if (threadIdx.x == 0) item_s = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= total) return;
        int lo = 0, hi = nviews - 1;       // last view with prefix[v] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const RenderArgs &a = views[lo];
        if (a.status->last_pairs > a.capacity) continue;   // that view overflowed
        const uint32_t ord = a.tile_order[item - prefix[lo]];
        const int tile = (int)(ord & kTileMask);
        if (use_tc(a) && !(ord & kTileWide))
            raster_tile_tc<false, false>(a, tile, sm.tc);
        else if (threadIdx.x < kThreads)
            raster_tile<false, false>(a, tile, sm.buf);
    }
}

template <bool kAux, bool kCount>
cudaError_t launch_t(const RenderArgs &a, cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    if (use_tc(a))
        k_raster_tc<kAux, kCount><<<T, kTcThreads, 0, stream>>>(a);
    else
        k_raster<kAux, kCount><<<T, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_raster(const RenderArgs &a, cudaStream_t stream) {
    const bool aux = a.out_aux != nullptr, cnt = a.out_count != nullptr;
    if (a.out_depth) {   // depth image (Eq. 5), no aux / count outputs
        if (use_tc(a))
            k_raster_tc<false, false, true><<<a.cam.tiles_x * a.cam.tiles_y, kTcThreads, 0, stream>>>(a);
        else
            k_raster<false, false, true><<<a.cam.tiles_x * a.cam.tiles_y, kThreads, 0, stream>>>(a);
        return cudaGetLastError();
    }
    if (aux && cnt) return launch_t<true, true>(a, stream);
    if (aux) return launch_t<true, false>(a, stream);
    if (cnt) return launch_t<false, true>(a, stream);
    return launch_t<false, false>(a, stream);
}

}  // namespace mgs

namespace mgs {

cudaError_t launch_raster_batch(const RenderArgs *views_dev, const int *prefix_dev, int nviews,
                                unsigned *counter_dev, int sm_count, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(counter_dev, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_batch, kTcThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_raster_batch<<<sm_count * per_sm, kTcThreads, 0, stream>>>(views_dev, prefix_dev, nviews,
                                                                 counter_dev);
    return cudaGetLastError();
}

}  // namespace mgs
