// Throughput probes (measurement support, not part of the render path): the
// two pipes that bound the rasteriser, ex2.approx.ftz.f32 (the MUFU / XU pipe;
// one per included pixel-Gaussian pair) and FP32 FFMA (the FMA pipe), and
// the rate of scattered 4-byte stores, one 32-byte sector each (what bounds
// the binning scatter, whose list entries each go to a different tile).
//
// Every block runs 256 threads with eight independent dependency chains each
// and records its SM and its first and last cycle on that SM's counter; per
// SM, the rate is the operations of the blocks it ran over the span from the
// earliest start to the latest end (whatever the blocks' residency), and the
// result is the mean over the SMs.
#include <algorithm>
#include <climits>
#include <vector>

#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kProbeIters = 2048;

__device__ __forceinline__ float probe_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kind 0: ex2 chains x -> ex2(x) (stays in (0, 1]); kind 1: FFMA chains.
template <int kKind>
__global__ void __launch_bounds__(kProbeThreads) k_probe(float *sink, long long *cycles) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = -0.001f * (float)(threadIdx.x + k);
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = kKind == 0 ? probe_ex2(a[k]) : fmaf(a[k], 0.999f, 1e-4f);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.f) sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;   // keeps the chains live
    if (threadIdx.x == 0) {
        cycles[3 * blockIdx.x] = (long long)smid;
        cycles[3 * blockIdx.x + 1] = t0;
        cycles[3 * blockIdx.x + 2] = t1;
    }
}

// Scattered stores: every lane writes 4 bytes to its own 32-byte sector of a
// 64 MB buffer (L2-resident, like the tile lists), kProbeStores per thread.
constexpr int kProbeStores = 256;
constexpr uint32_t kProbeWords = 16u << 20;
__global__ void __launch_bounds__(kProbeThreads) k_probe_store(uint32_t *buf, long long *cycles) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const uint32_t tid = blockIdx.x * kProbeThreads + threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    uint32_t h = tid * 2654435761u;
    for (int i = 0; i < kProbeStores; ++i) {
        h = h * 1664525u + 1013904223u;
        buf[(h >> 3) & (kProbeWords - 8u) & ~7u] = tid;   // sector start: 8 words per sector
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        cycles[3 * blockIdx.x] = (long long)smid;
        cycles[3 * blockIdx.x + 1] = t0;
        cycles[3 * blockIdx.x + 2] = t1;
    }
}

// Mean over the SMs of (ops of the blocks an SM ran) / (its earliest start to
// latest end), from the per-block records of a probe launch.
double per_sm_rate(const std::vector<long long> &h, int blocks, double ops_per_block) {
    std::vector<long long> lo(1024, LLONG_MAX), hi(1024, LLONG_MIN), nb(1024, 0);
    for (int b = 0; b < blocks; ++b) {
        const long long sm = h[3 * b];
        if (sm < 0 || sm >= 1024) continue;
        lo[sm] = std::min(lo[sm], h[3 * b + 1]);
        hi[sm] = std::max(hi[sm], h[3 * b + 2]);
        ++nb[sm];
    }
    double sum = 0.0;
    int used = 0;
    for (int sm = 0; sm < 1024; ++sm) {
        if (nb[sm] == 0 || hi[sm] <= lo[sm]) continue;
        sum += ops_per_block * (double)nb[sm] / (double)(hi[sm] - lo[sm]);
        ++used;
    }
    return used ? sum / used : 0.0;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_probe_store(int32_t device, double *sectors_per_sm_clk) {
    if (!sectors_per_sm_clk) {
        set_last_error("NULL argument");
        return MGS_ERR_INVALID_ARG;
    }
    int prev = -1, ndev = 0;
    // check the ordinal first: a failed cudaSetDevice would leave its error
    // for the next launch of this thread to report
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_last_error("no such CUDA device");
        return MGS_ERR_INVALID_ARG;
    }
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cannot select the device");
        return MGS_ERR_INVALID_ARG;
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * kProbeBlocksPerSm;
    uint32_t *buf = nullptr;
    long long *cyc = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)kProbeWords * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * 3 * sizeof(long long));
    double rate = 0.0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first run warms up
        k_probe_store<<<blocks, kProbeThreads>>>(buf, cyc);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess) {
        std::vector<long long> h((size_t)blocks * 3);
        e = cudaMemcpy(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) rate = per_sm_rate(h, blocks, (double)kProbeThreads * kProbeStores);
    }
    if (buf) cudaFree(buf);
    if (cyc) cudaFree(cyc);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MGS_ERR_CUDA;
    }
    *sectors_per_sm_clk = rate;
    return MGS_OK;
}

extern "C" mgs_status mgs_probe_rates(int32_t device, double *ex2_per_sm_clk,
                                      double *ffma_per_sm_clk) {
    if (!ex2_per_sm_clk || !ffma_per_sm_clk) {
        set_last_error("NULL argument");
        return MGS_ERR_INVALID_ARG;
    }
    int prev = -1, ndev = 0;
    // check the ordinal first: a failed cudaSetDevice would leave its error
    // for the next launch of this thread to report
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_last_error("no such CUDA device");
        return MGS_ERR_INVALID_ARG;
    }
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cannot select the device");
        return MGS_ERR_INVALID_ARG;
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * kProbeBlocksPerSm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)blocks * kProbeThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)blocks * 3 * sizeof(long long));
    double rate[2] = {0.0, 0.0};
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // first run warms up
            if (kind == 0) k_probe<0><<<blocks, kProbeThreads>>>(sink, cyc);
            else k_probe<1><<<blocks, kProbeThreads>>>(sink, cyc);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess) break;
        std::vector<long long> h((size_t)blocks * 3);
        e = cudaMemcpy(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        rate[kind] = per_sm_rate(h, blocks, (double)kProbeThreads * kProbeIters * 8);
    }
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MGS_ERR_CUDA;
    }
    *ex2_per_sm_clk = rate[0];
    *ffma_per_sm_clk = rate[1];
    return MGS_OK;
}
