// Load-time SH decode (Sec. 3.2, Eq. 6): every Gaussian stores a diffuse
// feature h_d and a view-dependent feature h_v (3 values each); two small
// MLPs with one hidden layer of 64 ReLU units and 16-bit parameters (App. C)
// turn them into the degree-0 and degree-1 SH coefficients once, before
// rendering:  f_d = MLP_d(h_d, h_v) -> Y0 rgb,  f_v = MLP_v(h_d, h_v) ->
// Y1 rgb, Y2 rgb, Y3 rgb.  One thread per Gaussian, FP32 accumulation, the
// parameters (passed by value) staged in shared memory as FP32.
#include <cuda_fp16.h>

#include <cstring>

#include "mgs_internal.cuh"

namespace mgs {
namespace {

constexpr int kDecThreads = 256;

struct DecodeParams {
    __half w1d[64 * 6], b1d[64], w2d[3 * 64], b2d[3];
    __half w1v[64 * 6], b1v[64], w2v[9 * 64], b2v[9];
};

struct DecodeSmem {
    float w1[2][64][6];
    float b1[2][64];
    float w2d[3][64], w2v[9][64];
    float b2[12];
};

template <bool kFP16>
__global__ void __launch_bounds__(kDecThreads)
    k_decode_sh(int64_t n, const void *__restrict__ h, void *__restrict__ attrs, DecodeParams p) {
    __shared__ DecodeSmem sm;
    for (int e = threadIdx.x; e < 64 * 6; e += blockDim.x) {
        sm.w1[0][e / 6][e % 6] = __half2float(p.w1d[e]);
        sm.w1[1][e / 6][e % 6] = __half2float(p.w1v[e]);
    }
    for (int e = threadIdx.x; e < 64; e += blockDim.x) {
        sm.b1[0][e] = __half2float(p.b1d[e]);
        sm.b1[1][e] = __half2float(p.b1v[e]);
    }
    for (int e = threadIdx.x; e < 3 * 64; e += blockDim.x) sm.w2d[e / 64][e % 64] = __half2float(p.w2d[e]);
    for (int e = threadIdx.x; e < 9 * 64; e += blockDim.x) sm.w2v[e / 64][e % 64] = __half2float(p.w2v[e]);
    if (threadIdx.x < 3) sm.b2[threadIdx.x] = __half2float(p.b2d[threadIdx.x]);
    if (threadIdx.x < 9) sm.b2[3 + threadIdx.x] = __half2float(p.b2v[threadIdx.x]);
    __syncthreads();

    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            x[k] = kFP16 ? __half2float(static_cast<const __half *>(h)[6 * i + k])
                         : static_cast<const float *>(h)[6 * i + k];
        float y[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = sm.b2[k];
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            float hd = sm.b1[0][j], hv = sm.b1[1][j];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                hd = fmaf(sm.w1[0][j][k], x[k], hd);
                hv = fmaf(sm.w1[1][j][k], x[k], hv);
            }
            hd = fmaxf(hd, 0.0f);
            hv = fmaxf(hv, 0.0f);
#pragma unroll
            for (int k = 0; k < 3; ++k) y[k] = fmaf(sm.w2d[k][j], hd, y[k]);
#pragma unroll
            for (int k = 0; k < 9; ++k) y[3 + k] = fmaf(sm.w2v[k][j], hv, y[3 + k]);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            if (kFP16)
                static_cast<__half *>(attrs)[kRec * i + 11 + k] = __float2half_rn(y[k]);
            else
                static_cast<float *>(attrs)[kRec * i + 11 + k] = y[k];
        }
    }
}

bool fill(const uint16_t *src, __half *dst, int count) {
    if (!src) return false;
    memcpy(dst, src, (size_t)count * 2);
    return true;
}

mgs_status bad(mgs_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace mgs

using namespace mgs;

extern "C" mgs_status mgs_decode_sh(mgs_ctx ctx, int64_t n, int32_t precision, const void *h,
                                    const mgs_sh_mlp *mlp_d, const mgs_sh_mlp *mlp_v,
                                    void *attrs, mgs_stream stream_) {
    if (!ctx || !mlp_d || !mlp_v) return bad(MGS_ERR_INVALID_ARG, "NULL argument");
    if (n < 0) return bad(MGS_ERR_INVALID_ARG, "n < 0");
    if (precision != MGS_PREC_FP32 && precision != MGS_PREC_FP16)
        return bad(MGS_ERR_INVALID_ARG, "unknown precision");
    if (n > 0 && (!h || !attrs)) return bad(MGS_ERR_INVALID_ARG, "h or attrs is NULL");
    DecodeParams p;
    if (!fill(mlp_d->w1, p.w1d, 64 * 6) || !fill(mlp_d->b1, p.b1d, 64) ||
        !fill(mlp_d->w2, p.w2d, 3 * 64) || !fill(mlp_d->b2, p.b2d, 3) ||
        !fill(mlp_v->w1, p.w1v, 64 * 6) || !fill(mlp_v->b1, p.b1v, 64) ||
        !fill(mlp_v->w2, p.w2v, 9 * 64) || !fill(mlp_v->b2, p.b2v, 9))
        return bad(MGS_ERR_INVALID_ARG, "an SH decoder parameter array is NULL");
    if (n == 0) return MGS_OK;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return bad(MGS_ERR_CUDA, "cannot select the context's device");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int64_t blocks = (n + kDecThreads - 1) / kDecThreads;
    const int64_t cap = (int64_t)ctx_sm_count(ctx) * 8;
    if (blocks > cap) blocks = cap;
    if (precision == MGS_PREC_FP16)
        k_decode_sh<true><<<(unsigned)blocks, kDecThreads, 0, stream>>>(n, h, attrs, p);
    else
        k_decode_sh<false><<<(unsigned)blocks, kDecThreads, 0, stream>>>(n, h, attrs, p);
    const cudaError_t e = cudaGetLastError();
    cudaSetDevice(prev);
    if (e != cudaSuccess) return bad(MGS_ERR_CUDA, "SH decode launch failed");
    return MGS_OK;
}
