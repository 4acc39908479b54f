// Spatial order of a resident scene.  At load time the Gaussians are sorted
// along a 3D Morton curve of their means (10 bits per axis over the scene's
// bounding box), so that Gaussians stored close together are close in space:
// a binning CTA's contiguous range of Gaussians then covers a compact set of
// tiles, and its list writes stay local.  The image does not depend on the
// storage order (Eq. 2 is a sum); every per-Gaussian output is mapped back to
// the caller's order through perm (stored position -> caller index) and its
// inverse.
#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kOrdThreads = 256;

// float <-> order-preserving unsigned encoding (for atomic min / max)
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

template <bool kFP16>
__device__ __forceinline__ void mean_of(const void *attrs, int64_t i, float (&m)[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        m[k] = kFP16 ? __half2float(static_cast<const __half *>(attrs)[kRec * i + k])
                     : static_cast<const float *>(attrs)[kRec * i + k];
}

// bounds[0..2] = min, bounds[3..5] = max of the finite means (encoded)
template <bool kFP16>
__global__ void __launch_bounds__(kOrdThreads) k_bounds(const void *attrs, int64_t n,
                                                        uint32_t *bounds) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float m[3];
        mean_of<kFP16>(attrs, i, m);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (isfinite(m[k])) {
                lo[k] = fminf(lo[k], m[k]);
                hi[k] = fmaxf(hi[k], m[k]);
            }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&bounds[k], f2ord(lo[k]));
            atomicMax(&bounds[3 + k], f2ord(hi[k]));
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {   // 10 bits -> every third bit
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

template <bool kFP16>
__global__ void __launch_bounds__(kOrdThreads) k_morton(const void *attrs, int64_t n,
                                                        const uint32_t *bounds, uint64_t *keys,
                                                        uint32_t *vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float m[3];
    mean_of<kFP16>(attrs, i, m);
    uint32_t key = 0x3FFFFFFFu;   // non-finite means last
    if (isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2])) {
        key = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float lo = ord2f(bounds[k]), hi = ord2f(bounds[3 + k]);
            const float ext = hi - lo;
            const float u = ext > 0.0f ? (m[k] - lo) / ext : 0.0f;
            const uint32_t q = (uint32_t)fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);
            key |= spread10(q) << k;
        }
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kOrdThreads) k_gather(const uint4 *__restrict__ in, int row16,
                                                        const uint32_t *__restrict__ order,
                                                        int64_t n, uint4 *__restrict__ out,
                                                        uint32_t *__restrict__ perm,
                                                        uint32_t *__restrict__ iperm) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t src = order[j];
    for (int k = 0; k < row16; ++k) out[j * row16 + k] = in[(int64_t)src * row16 + k];
    perm[j] = src;
    iperm[src] = (uint32_t)j;
}

__global__ void k_map_ids(const uint32_t *__restrict__ in, const uint32_t *__restrict__ perm,
                          int64_t k, uint32_t *__restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) out[j] = perm[in[j]];
}

template <class T>
cudaError_t alloc(T **p, size_t n) {
    return cudaMalloc(reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T));
}

}  // namespace

cudaError_t spatial_order(const void *attrs_in, int64_t n, int precision, void *attrs_out,
                          uint32_t *perm, uint32_t *iperm, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const bool fp16 = precision == MGS_PREC_FP16;
    uint64_t *k = nullptr, *kt = nullptr;
    uint32_t *v = nullptr, *vt = nullptr, *hist = nullptr, *bounds = nullptr;
    cudaError_t e = alloc(&k, (size_t)n);
    if (e == cudaSuccess) e = alloc(&kt, (size_t)n);
    if (e == cudaSuccess) e = alloc(&v, (size_t)n);
    if (e == cudaSuccess) e = alloc(&vt, (size_t)n);
    if (e == cudaSuccess) e = alloc(&hist, (size_t)sorted_hist_entries(n));
    if (e == cudaSuccess) e = alloc(&bounds, 6);
    const uint32_t init[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bounds, init, sizeof init, cudaMemcpyHostToDevice, stream);
    const unsigned grid = (unsigned)((n + kOrdThreads - 1) / kOrdThreads);
    if (e == cudaSuccess) {
        const unsigned gb = grid < 1024 ? grid : 1024;
        if (fp16)
            k_bounds<true><<<gb, kOrdThreads, 0, stream>>>(attrs_in, n, bounds);
        else
            k_bounds<false><<<gb, kOrdThreads, 0, stream>>>(attrs_in, n, bounds);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (fp16)
            k_morton<true><<<grid, kOrdThreads, 0, stream>>>(attrs_in, n, bounds, k, v);
        else
            k_morton<false><<<grid, kOrdThreads, 0, stream>>>(attrs_in, n, bounds, k, v);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = radix_sort(&k, &v, &kt, &vt, n, nullptr, 0, 32, hist, stream);
    if (e == cudaSuccess) {
        const int row16 = kRec * (fp16 ? 2 : 4) / 16;
        k_gather<<<grid, kOrdThreads, 0, stream>>>(static_cast<const uint4 *>(attrs_in), row16, v, n,
                                                   static_cast<uint4 *>(attrs_out), perm, iperm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(k);
    cudaFree(kt);
    cudaFree(v);
    cudaFree(vt);
    cudaFree(hist);
    cudaFree(bounds);
    return e;
}

cudaError_t map_ids(const uint32_t *in, const uint32_t *perm, int64_t count, uint32_t *out,
                    cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    k_map_ids<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(in, perm, count, out);
    return cudaGetLastError();
}

}  // namespace mgs
