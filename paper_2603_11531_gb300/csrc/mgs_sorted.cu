// Comparator: sorted front-to-back alpha blending (App. B, Eq. 11), the 3DGS
// compositing the paper removes (its "with sorting" baseline, Sec. 1 and
// Table 3).  Same preprocessing, same tile lists and the same inclusion test
// as the sort-free renderer; in addition every tile's list is ordered by view
// depth with a project-written radix sort, and each pixel blends front to back
//   C = sum_i c_i a_i T_i + T c_bg,  T_i = prod_{j<i} (1 - a_j),
// stopping before the Gaussian that would bring T below 1e-4 (3DGS early
// termination).
//
// Order: Gaussians are ranked by (FP32-contract view depth, caller index)
// with a stable radix sort of the depth bits over caller-ordered input; each
// tile's list (a segment of the counting sort's output) is then sorted by
// rank.  Both sorts are the CUDA library's (CUB) device radix / segmented
// sorts, the kind of sort a sorted 3DGS renderer uses, so the comparison is
// not made against a slow sort.  The project's own LSD radix sort below
// serves the load-time spatial order.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per block
constexpr int kRsBins = 16;                     // 4-bit digits

__device__ __forceinline__ int64_t count_of(int64_t n, const unsigned long long *n_dev) {
    if (!n_dev) return n;
    const unsigned long long d = *n_dev;
    return d < (unsigned long long)n ? (int64_t)d : n;
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t *__restrict__ keys,
                                                        int64_t n_max,
                                                        const unsigned long long *n_dev,
                                                        int shift, int nblocks,
                                                        uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kRsBins];
    const int64_t n = count_of(n_max, n_dev);
    if (threadIdx.x < kRsBins) h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (kRsBins - 1)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kRsBins) hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m uint32 values in place, one block.
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ v, int64_t m) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0u;
    __syncthreads();
    for (int64_t base = 0; base < m; base += 1024 * 4) {
        const int64_t i0 = base + (int64_t)tid * 4;
        uint32_t x[4], local = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[k] = (i0 + k < m) ? v[i0 + k] : 0u;
            local += x[k];
        }
        uint32_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        uint32_t run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < m) v[i0 + k] = run;
            run += x[k];
        }
        __syncthreads();
        if (tid == 1023) carry = run;
        __syncthreads();
    }
}

// Stable scatter of one 4-bit digit: thread t owns keys [8t, 8t + 8) of the
// block; ranks = global digit offset + counts of the digit in earlier threads
// + earlier keys of the same digit in this thread.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n_max,
    const unsigned long long *n_dev, int shift, int nblocks, const uint32_t *__restrict__ offs) {
    __shared__ uint32_t cnt[kRsBins * kRsThreads];
    __shared__ uint32_t warp_sums[kRsThreads / 32];
    const int64_t n = count_of(n_max, n_dev);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)tid * kRsItems;
    uint64_t k[kRsItems];
    uint32_t val[kRsItems];
    int d[kRsItems];
    uint32_t c[kRsBins];
#pragma unroll
    for (int b = 0; b < kRsBins; ++b) c[b] = 0u;
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const int64_t idx = base + i;
        if (idx < n) {
            k[i] = kin[idx];
            val[i] = vin[idx];
            d[i] = (int)((k[i] >> shift) & (kRsBins - 1));
#pragma unroll
            for (int b = 0; b < kRsBins; ++b) c[b] += (d[i] == b);
        } else {
            d[i] = -1;
        }
    }
    // digit-major layout [digit][thread]; scan it flat, then subtract the
    // digit's start to get the count of that digit in earlier threads
#pragma unroll
    for (int b = 0; b < kRsBins; ++b) cnt[b * kRsThreads + tid] = c[b];
    __syncthreads();
    // each thread scans 16 consecutive entries of the flat array
    uint32_t loc[kRsBins], sum = 0;
#pragma unroll
    for (int j = 0; j < kRsBins; ++j) {
        loc[j] = sum;
        sum += cnt[tid * kRsBins + j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kRsThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kRsThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t excl = incl - sum + (warp > 0 ? warp_sums[warp - 1] : 0u);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsBins; ++j) cnt[tid * kRsBins + j] = excl + loc[j];
    __syncthreads();
    uint32_t run[kRsBins];
#pragma unroll
    for (int b = 0; b < kRsBins; ++b) {
        const uint32_t start = cnt[b * kRsThreads];  // flat prefix at (digit b, thread 0)
        run[b] = offs[(int64_t)b * nblocks + blockIdx.x] + (cnt[b * kRsThreads + tid] - start);
    }
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        if (d[i] < 0) continue;
        uint32_t pos = 0;
#pragma unroll
        for (int b = 0; b < kRsBins; ++b)
            if (d[i] == b) pos = run[b]++;
        kout[pos] = k[i];
        vout[pos] = val[i];
    }
}

// Keys of the depth ranking: view depth bits (positive floats order as
// unsigned integers) in the high word, invisible Gaussians last.
// The input is laid out in caller order (j -> stored row iperm[j]), so the
// stable sort breaks depth ties by caller index.
__global__ void k_depth_keys(const ProjRec *__restrict__ rec, const uint2 *__restrict__ rect,
                             const uint32_t *__restrict__ iperm, int64_t n,
                             uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t i = iperm ? iperm[j] : (uint32_t)j;
    const uint2 r = rect[i];
    const bool vis = (r.x >> 16) > (r.x & 0xFFFF);
    keys[j] = vis ? __float_as_uint(rec[i].c.z) : 0xFFFFFFFFu;   // positive floats order as uints
    vals[j] = i;
}

__global__ void k_rank_scatter(const uint32_t *__restrict__ sorted_idx, int64_t n,
                               uint32_t *__restrict__ rank) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) rank[sorted_idx[j]] = (uint32_t)j;
}

// (tile, rank) keys of every list entry; one block per tile.
__global__ void k_tile_keys(const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ gids,
                            const uint32_t *__restrict__ rank, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals, const DevStatus *__restrict__ status,
                            uint64_t capacity) {
    if (status->last_pairs > capacity) return;
    const int t = blockIdx.x;
    for (uint32_t j = offsets[t] + threadIdx.x; j < offsets[t + 1]; j += blockDim.x) {
        const uint32_t g = gids[j];
        keys[j] = rank[g];
        vals[j] = g;
    }
}

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Front-to-back blending of each tile's depth-sorted list.  One CTA (two
// warps) per tile, warp = 16x8 block, lane = 4 pixels; candidates are culled
// per block exactly as in the sort-free rasteriser, in list (depth) order,
// and a warp stops once all its pixels have terminated.
template <bool kCount>
__global__ void __launch_bounds__(64) k_raster_sorted(RenderArgs args, const uint32_t *__restrict__ sorted) {
    __shared__ float4 buf[2][3][32];
    const DevCamera &cam = args.cam;
    const int tile = (int)(args.tile_order[blockIdx.x] & kTileMask);
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile, by0 = ty * kTile + 8 * warp;
    const int px0 = bx0 + 4 * (lane & 3);
    const int py = by0 + (lane >> 2);
    if (args.status->last_pairs > args.capacity) return;
    const uint32_t start = args.tile_offsets[tile];
    const uint32_t end = args.tile_offsets[tile + 1];
    const float bx = (float)bx0 + 8.0f, by = (float)by0 + 4.0f;
    const float pyc = (float)py + 0.5f;
    const float kq = -0.72134752044448170f;
    float C[4][3], T[4];
    int cnt[4];
    bool done[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        C[k][0] = C[k][1] = C[k][2] = 0.f;
        T[k] = 1.f;
        cnt[k] = 0;
        done[k] = (px0 + k >= cam.width) || (py >= cam.height);
    }
    float4(*wb)[32] = buf[warp];
    for (uint32_t base = start; base < end; base += 32) {
        const bool all_done = done[0] && done[1] && done[2] && done[3];
        if (__all_sync(0xffffffffu, all_done)) break;
        const uint32_t j = base + lane;
        bool cand = false;
        float4 a, b, c;
        if (j < end) {
            const uint32_t gid = __ldg(&sorted[j]);
            a = __ldg(&args.rec[gid].a);
            b = __ldg(&args.rec[gid].b);
            c = __ldg(&args.rec[gid].c);
            cand = block_may_hit(a.x, a.y, a.z, a.w, b.x, bx, by, 7.5f, 3.5f);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, cand);
        if (cand) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            const float iw = 1.0f / b.z;           // 1 / (-w)
            wb[0][pos] = a;
            wb[1][pos] = make_float4(b.x, b.y, b.w * iw, c.x * iw);   // l22, log2 o, c_r, c_g
            wb[2][pos] = make_float4(c.y * iw, 0.f, 0.f, 0.f);        // c_b
        }
        __syncwarp();
        const int nc = __popc(bal);
        for (int k = 0; k < nc; ++k) {
            const float4 s0 = wb[0][k], s1 = wb[1][k], s2 = wb[2][k];
            const float dy = __fsub_rn(pyc, s0.y);
            const float ldy = __fmul_rn(s0.w, dy);
            const float e2 = __fmul_rn(s1.x, dy);
            const float e2s = __fmul_rn(e2, e2);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const float dx = __fsub_rn((float)(px0 + p) + 0.5f, s0.x);
                const float e1 = __fmaf_rn(s0.z, dx, ldy);
                const float q = __fmaf_rn(e1, e1, e2s);
                if (done[p] || !(q <= 9.0f)) continue;
                const float al = fminf(ex2f(__fmaf_rn(q, kq, s1.y)), 0.99f);
                const float nt = T[p] * (1.0f - al);
                if (nt < 1e-4f) {
                    done[p] = true;
                    continue;
                }
                const float wgt = al * T[p];
                C[p][0] = fmaf(s1.z, wgt, C[p][0]);
                C[p][1] = fmaf(s1.w, wgt, C[p][1]);
                C[p][2] = fmaf(s2.x, wgt, C[p][2]);
                T[p] = nt;
                if (kCount) cnt[p] += 1;
            }
        }
        __syncwarp();
    }
    if (py >= cam.height) return;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int x = px0 + p;
        if (x >= cam.width) break;
        const int64_t q = (int64_t)py * cam.width + x;
        float *o = args.out_rgb + 3 * q;
        o[0] = fmaf(T[p], args.bg[0], C[p][0]);
        o[1] = fmaf(T[p], args.bg[1], C[p][1]);
        o[2] = fmaf(T[p], args.bg[2], C[p][2]);
        if (kCount) args.out_count[q] = cnt[p];
    }
}

}  // namespace

// Sorts (key, value) pairs by bits [begin_bit, end_bit) of the key (stable
// LSD, 4-bit digits).  n_max bounds the element count and sizes the grids;
// n_dev (nullable) holds the actual count on the device.  The result is in
// *k / *v (pointers swapped with the temporaries as needed).
cudaError_t radix_sort(uint64_t **k, uint32_t **v, uint64_t **kt, uint32_t **vt, int64_t n_max,
                       const unsigned long long *n_dev, int begin_bit, int end_bit,
                       uint32_t *hist, cudaStream_t stream) {
    if (n_max <= 1) return cudaSuccess;
    const int nblocks = (int)((n_max + kRsTile - 1) / kRsTile);
    for (int shift = begin_bit; shift < end_bit; shift += 4) {
        k_rs_hist<<<nblocks, kRsThreads, 0, stream>>>(*k, n_max, n_dev, shift, nblocks, hist);
        k_rs_scan<<<1, 1024, 0, stream>>>(hist, (int64_t)kRsBins * nblocks);
        k_rs_scatter<<<nblocks, kRsThreads, 0, stream>>>(*k, *v, *kt, *vt, n_max, n_dev, shift,
                                                          nblocks, hist);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::swap(*k, *kt);
        std::swap(*v, *vt);
    }
    return cudaSuccess;
}

int64_t sorted_hist_entries(int64_t n_max) { return kRsBins * ((n_max + kRsTile - 1) / kRsTile); }

size_t sorted_temp_bytes(int64_t n, int64_t capacity, int T) {
    size_t a = 0, b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, a, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                    (const uint32_t *)nullptr, (uint32_t *)nullptr, (int)n);
    cub::DeviceSegmentedSort::SortPairs(nullptr, b, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                        (const uint32_t *)nullptr, (uint32_t *)nullptr, (int)capacity,
                                        T, (const uint32_t *)nullptr, (const uint32_t *)nullptr);
    return a > b ? a : b;
}

cudaError_t launch_sorted(const RenderArgs &a, const SortedScratch &s, cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    cudaError_t e;
    size_t tb = s.temp_bytes;
    // 1. rank the Gaussians by (view depth, caller index): stable radix sort
    //    of the depth bits over caller-ordered input
    if (a.n > 0) {
        k_depth_keys<<<(unsigned)((a.n + 255) / 256), 256, 0, stream>>>(a.rec, a.rect, a.iperm, a.n,
                                                                         s.nkeys, s.nvals);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cub::DeviceRadixSort::SortPairs(s.temp, tb, s.nkeys, s.nkeys_tmp, s.nvals,
                                                 s.nvals_tmp, (int)a.n, 0, 32, stream)) != cudaSuccess)
            return e;
        k_rank_scatter<<<(unsigned)((a.n + 255) / 256), 256, 0, stream>>>(s.nvals_tmp, a.n, s.rank);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 2. order each tile's list (a segment of the binning output) by rank
    k_tile_keys<<<T, 128, 0, stream>>>(a.tile_offsets, a.gids, s.rank, s.keys, s.vals, a.status,
                                        a.capacity);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tb = s.temp_bytes;
    if ((e = cub::DeviceSegmentedSort::SortPairs(s.temp, tb, s.keys, s.keys_tmp, s.vals, s.vals_tmp,
                                                 (int)a.capacity, T, a.tile_offsets,
                                                 a.tile_offsets + 1, stream)) != cudaSuccess)
        return e;
    // 3. blend
    if (a.out_count)
        k_raster_sorted<true><<<T, 64, 0, stream>>>(a, s.vals_tmp);
    else
        k_raster_sorted<false><<<T, 64, 0, stream>>>(a, s.vals_tmp);
    return cudaGetLastError();
}

}  // namespace mgs
