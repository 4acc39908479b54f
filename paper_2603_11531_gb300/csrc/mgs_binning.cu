// Tile binning without any depth order.
//
// The paper removes depth sorting because the blending sums of Eq. 2 commute
// (Sec. 2, Eq. 1 discussion; Sec. 3.1).  The lists built here are keyed by
// tile only -- a counting sort by tile:
//
//   1. k_bin_count: CTA c owns a contiguous range of Gaussians and counts its
//      (tile, Gaussian) pairs into a shared-memory histogram over the tiles;
//      one global atomicAdd per (CTA, tile) reserves the CTA's block inside
//      the tile and returns its base.
//   2. k_scan: exclusive scan of the per-tile totals -> tile offsets.
//   3. k_bin_scatter: the same CTA re-expands its pairs and places each one at
//      offset[tile] + base[c][tile] + (shared-memory rank).
//
// Pairs are expanded warp-cooperatively: a warp's 32 Gaussians are flattened
// into one pair index space (prefix sum of rectangle areas) so a Gaussian
// covering thousands of tiles does not serialise one lane.  A pair is listed
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
    h = (int)(r.y >> 16) - y0;
}

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

// Calls f(tile, gid) for every (tile, Gaussian) pair of Gaussians
// [g0, g0 + 32) (one per lane) whose tile passes tile_may_hit, spreading the
// pairs of the rectangles over the warp's lanes.
template <class F>
__device__ __forceinline__ void warp_pairs(const uint2 *__restrict__ rect,
                                           const ProjRec *__restrict__ rec, int64_t n, int64_t g0,
                                           int tiles_x, F &&f) {
    const int lane = threadIdx.x & 31;
    const int64_t i = g0 + lane;
    int x0 = 0, y0 = 0, w = 0, h = 0;
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
    float gl22 = 0.f;
    if (i < n) {
        rect_of(rect[i], x0, y0, w, h);
        if (w > 0 && h > 0) {
            ga = rec[i].a;
            gl22 = rec[i].b.x;
        }
    }
    const int c = w * h;
    const float winv = w > 0 ? 1.0f / (float)w : 0.0f;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - c;
    const int P = __shfl_sync(0xffffffffu, incl, 31);
    for (int pb = 0; pb < P; pb += 32) {
        const int p = pb + lane;
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
        if (p < P) {
            const int k = p - oe;
            // k / ow via the reciprocal, then corrected by one step either way
            // (the product is off by at most 2^-23 (k + 0.5) / ow < 1 for any k < 2^23)
            int ky = (int)(((float)k + 0.5f) * oinv);
            if (ky * ow > k) --ky;
            else if ((ky + 1) * ow <= k) ++ky;
            const int tx = ox0 + (k - ky * ow), ty = oy0 + ky;
            if (tile_may_hit(mx, my, l11, l21, l22, tx, ty)) f(ty * tiles_x + tx, (uint32_t)(g0 + lo));
        }
    }
}

__device__ __forceinline__ void cta_range(int64_t n, int64_t &begin, int64_t &end) {
    const int64_t per = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
    begin = per * blockIdx.x;
    end = begin + per < n ? begin + per : n;
}

__global__ void __launch_bounds__(kBinThreads) k_bin_count(const uint2 *__restrict__ rect,
                                                           const ProjRec *__restrict__ rec,
                                                           int64_t n, int tiles_x, int T,
                                                           uint32_t *__restrict__ tile_count,
                                                           uint32_t *__restrict__ bases) {
    extern __shared__ uint32_t cnt_s[];
    int64_t begin, end;
    cta_range(n, begin, end);
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int band0 = 0; band0 < T; band0 += kBand) {
        const int bn = min(kBand, T - band0);
        for (int t = threadIdx.x; t < bn; t += blockDim.x) cnt_s[t] = 0u;
        __syncthreads();
        for (int64_t g0 = begin + 32 * warp; g0 < end; g0 += 32 * nwarps) {
            warp_pairs(rect, rec, end, g0, tiles_x, [&](int tile, uint32_t) {
                const int t = tile - band0;
                if ((unsigned)t < (unsigned)bn) atomicAdd(&cnt_s[t], 1u);
            });
        }
        __syncthreads();
        for (int t = threadIdx.x; t < bn; t += blockDim.x) {
            const uint32_t v = cnt_s[t];
            if (v) bases[(int64_t)blockIdx.x * T + band0 + t] = atomicAdd(&tile_count[band0 + t], v);
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

__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(
    const uint2 *__restrict__ rect, int64_t n, int tiles_x, int T,
    const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ bases,
    uint32_t *__restrict__ gids, uint64_t capacity, const DevStatus *__restrict__ status,
    const ProjRec *__restrict__ rec, uint4 *__restrict__ wt16) {
    extern __shared__ uint32_t cur_s[];
    if (status->last_pairs > capacity) return;  // overflow: lists are not built
    int64_t begin, end;
    cta_range(n, begin, end);
    if (wt16) {   // tensor-core rasteriser: FP16 weights of the visible Gaussians
        const int we = (int)((status->wmax_frame_bits >> 23) & 0xFFu) - 127;
        const float scale = we >= 14 ? __int_as_float((127 + 14 - we) << 23) : 1.0f;
        for (int64_t g = begin + threadIdx.x; g < end; g += blockDim.x) {
            const uint2 r = rect[g];
            if (r.x | r.y) wt16[g] = weights_f16(rec[g], scale);
        }
    }
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int band0 = 0; band0 < T; band0 += kBand) {
        const int bn = min(kBand, T - band0);
        // entries of tiles this CTA has no pairs in are never read
        for (int t = threadIdx.x; t < bn; t += blockDim.x)
            cur_s[t] = offsets[band0 + t] + bases[(int64_t)blockIdx.x * T + band0 + t];
        __syncthreads();
        for (int64_t g0 = begin + 32 * warp; g0 < end; g0 += 32 * nwarps) {
            warp_pairs(rect, rec, end, g0, tiles_x, [&](int tile, uint32_t gid) {
                const int t = tile - band0;
                if ((unsigned)t < (unsigned)bn) {
                    const uint32_t slot = atomicAdd(&cur_s[t], 1u);
                    if (slot < capacity) gids[slot] = gid;
                }
            });
        }
        __syncthreads();
    }
}

// Exclusive scan of tile_count[T] into tile_offsets[T+1], by one block; also
// records the pair count and flags capacity overflow.
__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t *__restrict__ count,
                                                       uint32_t *__restrict__ offsets, int T,
                                                       uint64_t capacity, DevStatus *status) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < T; base += kScanThreads * 4) {
        const int i0 = base + tid * 4;
        unsigned long long v[4], local = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < T) ? count[i0 + k] : 0u;
            local += v[k];
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
            unsigned long long s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
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
    }
}

// Rasterisation order: tiles by decreasing list length (bucketed by
// floor(log2(length))), so the longest tiles start first and the tail of the
// launch is made of short tiles.  One block.  Also hands this frame's weight
// bound to the rasteriser and resets the accumulator for the next frame.
__global__ void __launch_bounds__(kScanThreads) k_tile_order(const uint32_t *__restrict__ count,
                                                             int T, uint32_t *__restrict__ order,
                                                             DevStatus *status) {
    __shared__ uint32_t hist[33], start[33];
    const int tid = threadIdx.x;
    if (tid == 0) {
        status->wmax_frame_bits = status->wmax_bits;
        status->wmax_bits = 0u;
    }
    if (tid < 33) hist[tid] = 0u;
    __syncthreads();
    for (int t = tid; t < T; t += blockDim.x) {
        const uint32_t c = count[t];
        const int b = c ? 32 - __clz(c) : 0;      // 0 (empty) .. 32
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int b = 32; b >= 0; --b) {          // longest bucket first
            start[b] = run;
            run += hist[b];
        }
    }
    __syncthreads();
    for (int t = tid; t < T; t += blockDim.x) {
        const uint32_t c = count[t];
        const int b = c ? 32 - __clz(c) : 0;
        order[atomicAdd(&start[b], 1u)] = (uint32_t)t;
    }
}

}  // namespace

int bin_ctas(int64_t n, int sm_count) {
    int64_t c = (n + kBinThreads - 1) / kBinThreads;
    const int64_t cap = 2 * (int64_t)sm_count;
    if (c > cap) c = cap;
    return c < 1 ? 1 : (int)c;
}

cudaError_t launch_binning(const RenderArgs &a, int sm_count, uint32_t *bases,
                           cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    const int C = bin_ctas(a.n, sm_count);
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
        k_bin_count<<<C, kBinThreads, smem, stream>>>(a.rect, a.rec, a.n, a.cam.tiles_x, T,
                                                      a.tile_count, bases);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_scan<<<1, kScanThreads, 0, stream>>>(a.tile_count, a.tile_offsets, T, a.capacity, a.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_tile_order<<<1, kScanThreads, 0, stream>>>(a.tile_count, T, a.tile_order, a.status);
    if ((e = cudaGetLastError()) != cudaSuccess || a.n == 0) return e;
    k_bin_scatter<<<C, kBinThreads, smem, stream>>>(a.rect, a.n, a.cam.tiles_x, T, a.tile_offsets,
                                                    bases, a.gids, a.capacity, a.status, a.rec,
                                                    tc_raster(a) ? a.wt16 : nullptr);
    return cudaGetLastError();
}

}  // namespace mgs
