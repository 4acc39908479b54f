// Tile binning without any depth order.
//
// The paper removes depth sorting because the blending sums of Eq. 2 commute
// (Sec. 2, Eq. 1 discussion; Sec. 3.1).  The lists built here are keyed by
// tile only -- a counting sort by tile:
//
//   0. k_group_pairs, k_bin_plan: rectangle pair counts of every group of 32
//      consecutive Gaussians and the exclusive scan of the group costs (pairs
//      plus a fixed visit charge).  Every warp of the binning grid takes an
//      equal contiguous share of that cost numbering, so neither a warp nor
//      an SM waits on a few Gaussians that cover many tiles, nor on a long
//      stretch of Gaussians that cover almost none.
//   1. k_bin_count: each CTA counts the pairs of its warps' shares into a
//      shared-memory histogram over the tiles; one global atomicAdd per (CTA,
//      tile) reserves the CTA's block inside the tile and returns its base.
//   2. k_scan_order: exclusive scan of the per-tile totals -> tile offsets,
//      and the rasterisation order (longest lists first).
//   3. k_bin_scatter: the same CTA re-expands the same pairs and places each
//      one at offset[tile] + base[c][tile] + (shared-memory rank).
//
// Pairs are expanded warp-cooperatively: a group's 32 Gaussians are
// flattened into one pair index space (prefix sum of rectangle areas) so a
// Gaussian covering thousands of tiles does not serialise one lane.  A pair is listed
// only if the FP32 tile test (tile_may_hit) allows an included pixel in the
// tile; its rectangle alone (the 3-sigma bounding square) would list many
// tiles a thin ellipse never reaches.  Order within a
// tile follows the atomics and is not reproducible; the rasteriser does not
// depend on it beyond FP32 rounding.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kBinThreads = 1024;
constexpr int kBand = 32768;          // tiles per shared-memory band (128 KB)

__device__ __forceinline__ void rect_of(const uint2 r, int &x0, int &y0, int &w, int &h) {
    x0 = r.x & 0xFFFF;
    y0 = r.y & 0xFFFF;
    w = (int)(r.x >> 16) - x0;
    h = (int)((r.y & ~kRectWide) >> 16) - y0;
}
// Number of (tile, Gaussian) pairs of a rectangle.
__device__ __forceinline__ int rect_pairs(int w, int h) { return w > 0 && h > 0 ? w * h : 0; }

// FP32-contract tile test: may Gaussian (m, l) include a pixel centre of tile
// (tx, ty)?  Slab bounds at the tile centre with half extent 7.5 and a 2^-18
// relative margin, one correctly rounded operation per step (the oracle
// evaluates the identical sequence, so both build the same lists).  A tile
// that fails holds no pixel with q <= 9.
__device__ __forceinline__ bool tile_may_hit(float mx, float my, float l11, float l21, float l22,
                                             int tx, int ty) {
    const float h = 7.5f;
    const float bx = (float)(tx * kTile + 8), by = (float)(ty * kTile + 8);
    const float dxb = __fsub_rn(bx, mx);
    const float dyb = __fsub_rn(by, my);
    const float e1c = fabsf(__fmaf_rn(l11, dxb, __fmul_rn(l21, dyb)));
    const float h1 = __fmaf_rn(fabsf(l11), h, __fmul_rn(fabsf(l21), h));
    const float u2 = __fadd_rn(fabsf(dyb), h);
    const float s1 = __fadd_rn(__fmul_rn(fabsf(l11), __fadd_rn(fabsf(dxb), h)), __fmul_rn(fabsf(l21), u2));
    const float m1 = __fmul_rn(3.814697265625e-06f, __fadd_rn(s1, 4.0f));
    const float e2c = fabsf(__fmul_rn(l22, dyb));
    const float h2 = __fmul_rn(fabsf(l22), h);
    const float m2 = __fmul_rn(3.814697265625e-06f, __fadd_rn(__fmul_rn(fabsf(l22), u2), 4.0f));
    return __fsub_rn(e1c, h1) <= __fadd_rn(3.0f, m1) && __fsub_rn(e2c, h2) <= __fadd_rn(3.0f, m2);
}

// Calls f(tile, gid, wide) for the pairs [pa, pb) of the flattened pair
// numbering of Gaussians [g0, g0 + 32) (one per lane; rectangle after
// rectangle, row major inside each) whose tile passes tile_may_hit, 32 pairs
// at a time over the warp's lanes; wide = the Gaussian carries kRectWide.
// A lane's Gaussian of a group: rectangle and cull geometry, loaded together
// (the geometry of a Gaussian without a rectangle is loaded but never used),
// one group ahead of its use.
struct GroupLoad {
    uint2 r;
    float4 a;
    float l22;
};
__device__ __forceinline__ GroupLoad load_group(const uint2 *__restrict__ rect,
                                                const ProjRec *__restrict__ rec, int64_t n,
                                                int64_t g0) {
    GroupLoad L{make_uint2(0u, 0u), make_float4(0.f, 0.f, 0.f, 0.f), 0.f};
    const int64_t i = g0 + (threadIdx.x & 31);
    if (i < n) {
        L.r = __ldg(&rect[i]);
        L.a = __ldg(&rec[i].a);
        L.l22 = __ldg(&rec[i].b.x);
    }
    return L;
}

template <class F>
__device__ __forceinline__ void warp_pairs(const GroupLoad &L, int64_t g0, int tiles_x, int pa,
                                           int pb, F &&f) {
    const int lane = threadIdx.x & 31;
    int x0 = 0, y0 = 0, w = 0, h = 0;
    rect_of(L.r, x0, y0, w, h);
    const bool wide = (L.r.y & kRectWide) != 0;
    const float4 ga = L.a;
    const float gl22 = L.l22;
    const int c = rect_pairs(w, h);
    const float winv = w > 0 ? 1.0f / (float)w : 0.0f;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - c;
    const int P = min(__shfl_sync(0xffffffffu, incl, 31), pb);
    for (int base = pa; base < P; base += 32) {
        const int p = base + lane;
        // owner: the largest lane whose exclusive prefix is <= p
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(0xffffffffu, excl, lo + step);
            if (e <= p) lo += step;
        }
        const int ox0 = __shfl_sync(0xffffffffu, x0, lo);
        const int oy0 = __shfl_sync(0xffffffffu, y0, lo);
        const int ow = __shfl_sync(0xffffffffu, w, lo);
        const float oinv = __shfl_sync(0xffffffffu, winv, lo);
        const int oe = __shfl_sync(0xffffffffu, excl, lo);
        const float mx = __shfl_sync(0xffffffffu, ga.x, lo);
        const float my = __shfl_sync(0xffffffffu, ga.y, lo);
        const float l11 = __shfl_sync(0xffffffffu, ga.z, lo);
        const float l21 = __shfl_sync(0xffffffffu, ga.w, lo);
        const float l22 = __shfl_sync(0xffffffffu, gl22, lo);
        const bool owide = __shfl_sync(0xffffffffu, wide, lo);
        if (p < P) {
            const int k = p - oe;
            // k / ow via the reciprocal, then corrected by one step either way
            // (the product is off by at most 2^-23 (k + 0.5) / ow < 1 for any k < 2^23)
            int ky = (int)(((float)k + 0.5f) * oinv);
            if (ky * ow > k) --ky;
            else if ((ky + 1) * ow <= k) ++ky;
            const int tx = ox0 + (k - ky * ow), ty = oy0 + ky;
            if (tile_may_hit(mx, my, l11, l21, l22, tx, ty))
                f(ty * tiles_x + tx, (uint32_t)(g0 + lo), owide);
        }
    }
}

// Cost of a group in the work plan: its rectangle pairs plus a fixed charge
// for visiting it (loading and scanning 32 rectangles), so that shares over
// sparse stretches of the scene (many Gaussians, few pairs) stay short.
constexpr int kGroupCost = 64;

// Largest group g with cexcl[g] <= c (c < cexcl[groups]).
__device__ __forceinline__ int64_t find_group(const unsigned long long *__restrict__ cexcl,
                                              int64_t groups, unsigned long long c) {
    int64_t lo = 0, hi = groups - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cexcl[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Calls f(tile, gid, wide) for the listed pairs of this warp's share of the work
// plan: group g occupies costs [cexcl[g], cexcl[g + 1]), its visit charge
// first and then one unit per rectangle pair in the group's pair numbering;
// warp w of W takes costs [C w / W, C (w + 1) / W) of the total C.
template <class F>
__device__ __forceinline__ void warp_share_pairs(const uint2 *__restrict__ rect,
                                                 const ProjRec *__restrict__ rec, int64_t n,
                                                 const unsigned long long *__restrict__ cexcl,
                                                 int64_t groups, int tiles_x, F &&f) {
    if (groups == 0) return;
    const unsigned long long C = cexcl[groups];
    const unsigned long long W = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned long long c0 = C * w / W, c1 = C * (w + 1) / W;
    if (c0 >= c1) return;
    int64_t g = find_group(cexcl, groups, c0);
    unsigned long long e0 = cexcl[g];
    GroupLoad cur = load_group(rect, rec, n, g * 32);
    for (;;) {
        const unsigned long long e1 = cexcl[g + 1];
        const long long np = (long long)(e1 - e0) - kGroupCost;    // pairs of group g
        const long long pa = max(0ll, (long long)(c0 > e0 ? c0 - e0 : 0ull) - kGroupCost);
        const long long pb = min(np, (long long)(c1 - e0) - kGroupCost);
        const bool more = !(c1 <= e1 || g + 1 >= groups);
        GroupLoad nxt{};
        if (more) nxt = load_group(rect, rec, n, (g + 1) * 32);   // in flight meanwhile
        if (pa < pb) warp_pairs(cur, g * 32, tiles_x, (int)pa, (int)pb, f);
        if (!more) break;
        ++g;
        e0 = e1;
        cur = nxt;
    }
}

// Rectangle pair count of every group of 32 consecutive Gaussians (one warp
// per group).
__global__ void __launch_bounds__(kBinThreads) k_group_pairs(const uint2 *__restrict__ rect,
                                                             int64_t n, uint32_t *__restrict__ grp) {
    const int64_t g = ((int64_t)blockIdx.x * kBinThreads + threadIdx.x) >> 5;
    const int64_t i = g * 32 + (threadIdx.x & 31);
    uint32_t c = 0;
    if (i < n) {
        int x0, y0, w, h;
        rect_of(rect[i], x0, y0, w, h);
        c = (uint32_t)rect_pairs(w, h);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && g * 32 < n) grp[g] = c;
}

// Exclusive scan of the group costs (pairs + kGroupCost) into
// cexcl[0..groups] (64-bit), by one block, kPlanSeg groups at a time staged
// in shared memory so that global loads and stores stay coalesced.
constexpr int kPlanSeg = 16384;   // 64-bit costs per pass
// Shared-memory slot of entry i: one pad word every 16 entries, so that
// threads scanning runs of 16 consecutive entries hit different banks.
__device__ __forceinline__ int plan_slot(int i) { return i + (i >> 4); }
constexpr int kPlanSlots = kPlanSeg + kPlanSeg / 16;
__global__ void __launch_bounds__(kScanThreads) k_bin_plan(const uint32_t *__restrict__ grp,
                                                           int64_t groups,
                                                           unsigned long long *__restrict__ cexcl) {
    extern __shared__ unsigned long long seg[];
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long carry = 0;   // identical in every thread
    for (int64_t s0 = 0; s0 < groups; s0 += kPlanSeg) {
        const int m = (int)(groups - s0 < kPlanSeg ? groups - s0 : kPlanSeg);
        for (int i = tid; i < m; i += kScanThreads)
            seg[plan_slot(i)] = (unsigned long long)grp[s0 + i] + kGroupCost;
        __syncthreads();
        const int per = (m + kScanThreads - 1) / kScanThreads;
        const int lo = min(tid * per, m), hi = min(lo + per, m);
        unsigned long long local = 0;
        for (int i = lo; i < hi; ++i) local += seg[plan_slot(i)];
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_sums[lane] = t;
        }
        __syncthreads();
        unsigned long long run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0ull);
        for (int i = lo; i < hi; ++i) {
            const unsigned long long v = seg[plan_slot(i)];
            seg[plan_slot(i)] = run;
            run += v;
        }
        carry += warp_sums[kScanThreads / 32 - 1];
        __syncthreads();
        for (int i = tid; i < m; i += kScanThreads) cexcl[s0 + i] = seg[plan_slot(i)];
        __syncthreads();
    }
    if (tid == 0) cexcl[groups] = carry;
}

// Counts per tile; with `tc` (tensor-core rasteriser) and a frame that has
// wide Gaussians, also sets kTileWide in tile_count[] of every tile that
// lists one (per-CTA counts stay below 2^31, so the flag never meets a carry).
__global__ void __launch_bounds__(kBinThreads, 1) k_bin_count(const uint2 *__restrict__ rect,
                                                           const ProjRec *__restrict__ rec,
                                                           int64_t n, int tiles_x, int T,
                                                           const unsigned long long *__restrict__ excl,
                                                           int64_t groups,
                                                           uint32_t *__restrict__ tile_count,
                                                           uint32_t *__restrict__ bases,
                                                           const DevStatus *__restrict__ status,
                                                           bool tc) {
    extern __shared__ uint32_t cnt_s[];
    const bool mark = tc && status->wide_bits != 0u;
    for (int band0 = 0; band0 < T; band0 += kBand) {
        const int bn = min(kBand, T - band0);
        for (int t = threadIdx.x; t < bn; t += blockDim.x) cnt_s[t] = 0u;
        __syncthreads();
        warp_share_pairs(rect, rec, n, excl, groups, tiles_x, [&](int tile, uint32_t, bool wide) {
            const int t = tile - band0;
            if ((unsigned)t < (unsigned)bn) {
                atomicAdd(&cnt_s[t], 1u);
                if (mark && wide) atomicOr(&cnt_s[t], kTileWide);
            }
        });
        __syncthreads();
        for (int t = threadIdx.x; t < bn; t += blockDim.x) {
            const uint32_t v = cnt_s[t];
            const uint32_t c = v & kTileMask;
            if (c)
                bases[(int64_t)blockIdx.x * T + band0 + t] =
                    atomicAdd(&tile_count[band0 + t], c) & kTileMask;
            if (v & kTileWide) atomicOr(&tile_count[band0 + t], kTileWide);
        }
        __syncthreads();
    }
}

// Tensor-core weights of Gaussian g: (w c_r, w c_g, w c_b, w) times the
// frame's power-of-two scale (2^(14 - e) when the largest weight has
// exponent e >= 14), as FP16 high parts then FP16 low parts.
__device__ __forceinline__ uint4 weights_f16(const ProjRec &r, float scale) {
    const float w[4] = {-r.b.w * scale, -r.c.x * scale, -r.c.y * scale, -r.b.z * scale};
    __half hi[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        hi[k] = __float2half_rn(w[k]);
        lo[k] = __float2half_rn(w[k] - __half2float(hi[k]));
    }
    uint4 u;
    u.x = (uint32_t)__half_as_ushort(hi[0]) | ((uint32_t)__half_as_ushort(hi[1]) << 16);
    u.y = (uint32_t)__half_as_ushort(hi[2]) | ((uint32_t)__half_as_ushort(hi[3]) << 16);
    u.z = (uint32_t)__half_as_ushort(lo[0]) | ((uint32_t)__half_as_ushort(lo[1]) << 16);
    u.w = (uint32_t)__half_as_ushort(lo[2]) | ((uint32_t)__half_as_ushort(lo[3]) << 16);
    return u;
}

__global__ void __launch_bounds__(kBinThreads, 1) k_bin_scatter(
    const uint2 *__restrict__ rect, int64_t n, int tiles_x, int T,
    const unsigned long long *__restrict__ excl, int64_t groups,
    const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ bases,
    uint32_t *__restrict__ gids, uint64_t capacity, const DevStatus *__restrict__ status,
    const ProjRec *__restrict__ rec, uint4 *__restrict__ wt16) {
    extern __shared__ uint32_t cur_s[];
    if (status->last_pairs > capacity) return;  // overflow: lists are not built
    if (wt16) {   // tensor-core rasteriser: FP16 weights of the visible Gaussians
        const int we = (int)((status->wmax_frame_bits >> 23) & 0xFFu) - 127;
        const float scale = we >= 14 ? __int_as_float((127 + 14 - we) << 23) : 1.0f;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
             g += (int64_t)gridDim.x * blockDim.x) {
            const uint2 r = rect[g];
            if (r.x | r.y) wt16[g] = weights_f16(rec[g], scale);
        }
    }
    for (int band0 = 0; band0 < T; band0 += kBand) {
        const int bn = min(kBand, T - band0);
        // entries of tiles this CTA has no pairs in are never read
        for (int t = threadIdx.x; t < bn; t += blockDim.x)
            cur_s[t] = offsets[band0 + t] + bases[(int64_t)blockIdx.x * T + band0 + t];
        __syncthreads();
        warp_share_pairs(rect, rec, n, excl, groups, tiles_x, [&](int tile, uint32_t gid, bool) {
            const int t = tile - band0;
            if ((unsigned)t < (unsigned)bn) {
                const uint32_t slot = atomicAdd(&cur_s[t], 1u);
                if (slot < capacity) gids[slot] = gid;
            }
        });
        __syncthreads();
    }
}

// One block over the per-tile totals:
//   * exclusive scan of tile_count[T] into tile_offsets[T+1]; records the
//     pair count and flags capacity overflow;
//   * rasterisation order: tiles by decreasing list length (bucketed by
//     floor(log2(length))), so the longest tiles start first and the tail of
//     the raster launch is made of short tiles;
//   * hands this frame's weight bound to the rasteriser and resets the
//     accumulator (and the wide-Gaussian flag) for the next frame;
//   * carries each tile's kTileWide flag from tile_count[] into its order
//     entry.
__global__ void __launch_bounds__(kScanThreads) k_scan_order(const uint32_t *__restrict__ count,
                                                             uint32_t *__restrict__ offsets,
                                                             uint32_t *__restrict__ order, int T,
                                                             uint64_t capacity, DevStatus *status) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    __shared__ unsigned long long carry;
    __shared__ uint32_t hist[33], start[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry = 0;
        status->wmax_frame_bits = status->wmax_bits;
        status->wmax_bits = 0u;
        status->wide_bits = 0u;
        status->last_visible = status->visible;
        status->visible = 0u;
        status->last_wide_tiles = 0u;
    }
    if (tid < 33) hist[tid] = 0u;
    __syncthreads();
    for (int base = 0; base < T; base += kScanThreads * 4) {
        const int i0 = base + tid * 4;
        unsigned long long v[4], local = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < T) ? (count[i0 + k] & kTileMask) : 0u;
            local += v[k];
            if (i0 + k < T) {
                const uint32_t c = (uint32_t)v[k];
                atomicAdd(&hist[c ? 32 - __clz(c) : 0], 1u);   // bucket 0 (empty) .. 32
            }
        }
        unsigned long long incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long sw = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, sw, o);
                if (lane >= o) sw += y;
            }
            warp_sums[lane] = sw;
        }
        __syncthreads();
        unsigned long long run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0ull);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < T) offsets[i0 + k] = (uint32_t)run;
            run += v[k];
        }
        __syncthreads();
        if (tid == kScanThreads - 1) carry = run;
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long K = carry;
        offsets[T] = (uint32_t)K;
        status->last_pairs = K;
        atomicMax(&status->max_pairs, K);
        if (K > capacity || K > 0xFFFFFFFFull) atomicOr(&status->overflow, kStatusOverflow);
        uint32_t r = 0;
        for (int bk = 32; bk >= 0; --bk) {      // longest bucket first
            start[bk] = r;
            r += hist[bk];
        }
    }
    __syncthreads();
    for (int t = tid; t < T; t += blockDim.x) {
        const uint32_t cw = count[t], c = cw & kTileMask;
        order[atomicAdd(&start[c ? 32 - __clz(c) : 0], 1u)] = (uint32_t)t | (cw & kTileWide);
        if (cw & kTileWide) atomicAdd(&status->last_wide_tiles, 1u);
    }
}

}  // namespace

// One 1024-thread CTA per SM at most: the work plan balances the warps, so a
// second resident CTA would only add per-CTA tile bases.
int bin_ctas(int64_t n, int sm_count) {
    int64_t c = (n + kBinThreads - 1) / kBinThreads;
    const int64_t cap = (int64_t)sm_count;
    if (c > cap) c = cap;
    return c < 1 ? 1 : (int)c;
}

int64_t bin_scratch_words(int64_t n, int64_t T, int sm_count) {
    return bin_scratch_words_for(bin_ctas(n, sm_count), T, n);
}

cudaError_t launch_binning(const RenderArgs &a, int sm_count, uint32_t *scratch,
                           cudaStream_t stream, const cudaEvent_t *marks) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    const int C = bin_ctas(a.n, sm_count);
    const int64_t groups = (a.n + 31) / 32;
    uint32_t *bases = scratch;
    unsigned long long *excl =
        reinterpret_cast<unsigned long long *>(scratch + ((int64_t)C * T + 1) / 2 * 2);
    uint32_t *grp = reinterpret_cast<uint32_t *>(excl + groups + 1);
    const size_t smem = (size_t)(T < kBand ? T : kBand) * sizeof(uint32_t);
    cudaError_t e = cudaMemsetAsync(a.tile_count, 0, (size_t)T * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    if (a.n > 0) {
        if ((e = cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kBand * sizeof(uint32_t)))) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kBand * sizeof(uint32_t)))) != cudaSuccess)
            return e;
        k_group_pairs<<<(int)((groups * 32 + kBinThreads - 1) / kBinThreads), kBinThreads, 0,
                        stream>>>(a.rect, a.n, grp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int plan_n = (int)(groups < kPlanSeg ? groups : kPlanSeg);
        const size_t plan_smem = (size_t)(plan_n + plan_n / 16) * sizeof(unsigned long long);
        if ((e = cudaFuncSetAttribute(k_bin_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kPlanSlots * sizeof(unsigned long long)))) != cudaSuccess)
            return e;
        k_bin_plan<<<1, kScanThreads, plan_smem, stream>>>(grp, groups, excl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (marks && (e = cudaEventRecord(marks[0], stream)) != cudaSuccess) return e;
        k_bin_count<<<C, kBinThreads, smem, stream>>>(a.rect, a.rec, a.n, a.cam.tiles_x, T, excl,
                                                      groups, a.tile_count, bases, a.status,
                                                      tc_raster(a));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (marks && (e = cudaEventRecord(marks[1], stream)) != cudaSuccess) return e;
    } else if (marks) {
        if ((e = cudaEventRecord(marks[0], stream)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(marks[1], stream)) != cudaSuccess) return e;
    }
    k_scan_order<<<1, kScanThreads, 0, stream>>>(a.tile_count, a.tile_offsets, a.tile_order, T,
                                                 a.capacity, a.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (marks && (e = cudaEventRecord(marks[2], stream)) != cudaSuccess) return e;
    if (a.n == 0) return e;
    k_bin_scatter<<<C, kBinThreads, smem, stream>>>(a.rect, a.n, a.cam.tiles_x, T, excl, groups,
                                                    a.tile_offsets, bases, a.gids, a.capacity,
                                                    a.status, a.rec, tc_raster(a) ? a.wt16 : nullptr);
    return cudaGetLastError();
}

}  // namespace mgs
