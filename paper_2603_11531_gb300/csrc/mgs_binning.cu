// Tile binning without any depth order.
//
// The paper removes depth sorting because the blending sums of Eq. 2 commute
// (Sec. 2, Eq. 1 discussion; Sec. 3.1).  The lists built here are keyed by
// tile only: per-tile counts (accumulated by preprocessing) -> exclusive scan
// -> scatter of each Gaussian index into every tile of its rectangle.  A
// tile's list order is whatever order the scatter produced; the rasteriser
// does not depend on it beyond FP32 rounding.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kScanThreads = 1024;

// Exclusive scan of tile_count[T] into tile_offsets[T+1] and tile_cursor[T],
// by one block.  Also records the pair count and flags capacity overflow.
__global__ void __launch_bounds__(kScanThreads) k_scan(const uint32_t *__restrict__ count,
                                                       uint32_t *__restrict__ offsets,
                                                       uint32_t *__restrict__ cursor, int T,
                                                       uint64_t capacity, DevStatus *status) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < T; base += kScanThreads * 4) {
        // each thread owns 4 consecutive tiles of this chunk
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
            warp_sums[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        unsigned long long run = carry + (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0ull);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < T) {
                offsets[i0 + k] = (uint32_t)run;
                cursor[i0 + k] = (uint32_t)run;
            }
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
        if (K > capacity || K > 0xFFFFFFFFull) atomicOr(&status->overflow, 1u);
    }
}

// Scatter: Gaussian i is appended to every tile of its rectangle.
__global__ void __launch_bounds__(256) k_scatter(const uint2 *__restrict__ rect, int64_t n,
                                                 int tiles_x, uint32_t *__restrict__ cursor,
                                                 uint32_t *__restrict__ gids, uint64_t capacity,
                                                 const DevStatus *__restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (status->last_pairs > capacity) return;
    const uint2 r = rect[i];
    const int x0 = r.x & 0xFFFF, x1 = r.x >> 16, y0 = r.y & 0xFFFF, y1 = r.y >> 16;
    for (int ty = y0; ty < y1; ++ty)
        for (int tx = x0; tx < x1; ++tx) {
            const uint32_t slot = atomicAdd(&cursor[ty * tiles_x + tx], 1u);
            if (slot < capacity) gids[slot] = (uint32_t)i;
        }
}

}  // namespace

cudaError_t launch_binning(const RenderArgs &a, cudaStream_t stream) {
    const int T = a.cam.tiles_x * a.cam.tiles_y;
    k_scan<<<1, kScanThreads, 0, stream>>>(a.tile_count, a.tile_offsets, a.tile_cursor, T,
                                           a.capacity, a.status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.n == 0) return e;
    const int64_t blocks = (a.n + 255) / 256;
    k_scatter<<<(unsigned)blocks, 256, 0, stream>>>(a.rect, a.n, a.cam.tiles_x, a.tile_cursor,
                                                    a.gids, a.capacity, a.status);
    return cudaGetLastError();
}

}  // namespace mgs
