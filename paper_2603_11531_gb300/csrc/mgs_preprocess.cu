// Preprocessing: one thread per Gaussian.
//
//   App. B   projection of mu, EWA 2D covariance (3DGS convention),
//   Sec. 3.1 camera-Gaussian vector P_i = (mu_i - t_v) / |mu_i - t_v|,
//   Sec. 3.2 first-order SH colour,
//   Eq. 4    enhancement MLP (BF16 tensor cores, FP32 accumulation),
//   Eq. 3    depth-aware weight w_i,
// plus the tile rectangle used by binning.
//
// Visibility, the tile rectangle and the inclusion-test factors follow a fixed
// sequence of correctly rounded FP32 operations (no contraction, explicit
// fma), so that every IEEE-754 implementation of the sequence produces the same
// bits.  Colour, MLP and weight are ordinary FP32 values.
#include "mgs_internal.cuh"
#include "mgs_mlp.cuh"
#include "mgs_tcgen05.cuh"

namespace mgs {
namespace {

constexpr int kThreads = 128;  // 4 warps; each warp runs the MLP on 32 rows

__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float f_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float f_sqrt(float a) { return __fsqrt_rn(a); }

template <bool kFP16>
__device__ __forceinline__ void load_record(const void *attrs, int64_t i, float (&v)[kRec]) {
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

// Normalised quaternion (FP32 contract).  Returns false for a zero quaternion.
__device__ __forceinline__ bool contract_quat(const float (&v)[kRec], float &w, float &x,
                                              float &y, float &z) {
    const float qw = v[6], qx = v[7], qy = v[8], qz = v[9];
    float n2 = f_fma(qw, qw, f_fma(qx, qx, f_fma(qy, qy, f_mul(qz, qz))));
    float qn = f_sqrt(n2);
    w = f_div(qw, qn);
    x = f_div(qx, qn);
    y = f_div(qy, qn);
    z = f_div(qz, qn);
    return n2 > 0.0f;
}

struct Contract {
    bool visible;
    int rect[4];   // x_lo, y_lo, x_hi, y_hi
    float mx, my, l11, l21, l22, tz;
};

// Projection, EWA covariance, rectangle and inclusion factors (FP32 contract).
__device__ __forceinline__ Contract contract_project(const float (&v)[kRec], float w, float x,
                                                     float y, float z, bool qok,
                                                     const DevCamera &cam) {
    Contract o;
    o.visible = false;
    o.rect[0] = o.rect[1] = o.rect[2] = o.rect[3] = 0;
    o.mx = o.my = o.l11 = o.l21 = o.l22 = 0.0f;
    const float mux = v[0], muy = v[1], muz = v[2];
    const float s[3] = {v[3], v[4], v[5]};
    const float *W = cam.R;

    float xx = f_mul(x, x), yy = f_mul(y, y), zz = f_mul(z, z);
    float xy = f_mul(x, y), xz = f_mul(x, z), yz = f_mul(y, z);
    float wx = f_mul(w, x), wy = f_mul(w, y), wz = f_mul(w, z);
    float R[9];
    R[0] = f_sub(1.0f, f_mul(2.0f, f_add(yy, zz)));
    R[1] = f_mul(2.0f, f_sub(xy, wz));
    R[2] = f_mul(2.0f, f_add(xz, wy));
    R[3] = f_mul(2.0f, f_add(xy, wz));
    R[4] = f_sub(1.0f, f_mul(2.0f, f_add(xx, zz)));
    R[5] = f_mul(2.0f, f_sub(yz, wx));
    R[6] = f_mul(2.0f, f_sub(xz, wy));
    R[7] = f_mul(2.0f, f_add(yz, wx));
    R[8] = f_sub(1.0f, f_mul(2.0f, f_add(xx, yy)));

    float tx = f_fma(W[0], mux, f_fma(W[1], muy, f_fma(W[2], muz, cam.t[0])));
    float ty = f_fma(W[3], mux, f_fma(W[4], muy, f_fma(W[5], muz, cam.t[1])));
    float tz = f_fma(W[6], mux, f_fma(W[7], muy, f_fma(W[8], muz, cam.t[2])));
    o.tz = tz;
    if (!qok || !(tz > cam.znear)) return o;

    float rz = f_div(1.0f, tz);
    float txz = f_mul(tx, rz), tyz = f_mul(ty, rz);
    float limx = f_mul(1.3f, f_div(f_mul(0.5f, (float)cam.width), cam.fx));
    float limy = f_mul(1.3f, f_div(f_mul(0.5f, (float)cam.height), cam.fy));
    float txc = fminf(fmaxf(txz, -limx), limx);
    float tyc = fminf(fmaxf(tyz, -limy), limy);
    float J00 = f_mul(cam.fx, rz), J02 = -f_mul(f_mul(cam.fx, txc), rz);
    float J11 = f_mul(cam.fy, rz), J12 = -f_mul(f_mul(cam.fy, tyc), rz);

    float T0[3], T1[3], M[9], V0[3], V1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T0[j] = f_fma(J02, W[6 + j], f_mul(J00, W[j]));
        T1[j] = f_fma(J12, W[6 + j], f_mul(J11, W[3 + j]));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * k + j] = f_mul(R[3 * k + j], s[j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        V0[j] = f_fma(T0[2], M[6 + j], f_fma(T0[1], M[3 + j], f_mul(T0[0], M[j])));
        V1[j] = f_fma(T1[2], M[6 + j], f_fma(T1[1], M[3 + j], f_mul(T1[0], M[j])));
    }
    float ca = f_add(f_fma(V0[0], V0[0], f_fma(V0[1], V0[1], f_mul(V0[2], V0[2]))), 0.3f);
    float cb = f_fma(V0[0], V1[0], f_fma(V0[1], V1[1], f_mul(V0[2], V1[2])));
    float cc = f_add(f_fma(V1[0], V1[0], f_fma(V1[1], V1[1], f_mul(V1[2], V1[2]))), 0.3f);
    float det = f_fma(ca, cc, -f_mul(cb, cb));
    if (!(det > 0.0f)) return o;

    float mx = f_fma(cam.fx, txz, cam.cx);
    float my = f_fma(cam.fy, tyz, cam.cy);

    float mid = f_mul(0.5f, f_add(ca, cc));
    float hd = f_mul(0.5f, f_sub(ca, cc));
    float lam = f_add(mid, f_sqrt(f_fma(hd, hd, f_mul(cb, cb))));
    float rad = ceilf(f_mul(3.0f, f_sqrt(lam)));
    float vv[4];
    vv[0] = floorf(f_mul(f_sub(mx, rad), 0.0625f));
    vv[1] = floorf(f_mul(f_sub(my, rad), 0.0625f));
    vv[2] = f_add(floorf(f_mul(f_add(mx, rad), 0.0625f)), 1.0f);
    vv[3] = f_add(floorf(f_mul(f_add(my, rad), 0.0625f)), 1.0f);
    const float lim[4] = {(float)cam.tiles_x, (float)cam.tiles_y, (float)cam.tiles_x,
                          (float)cam.tiles_y};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float c = vv[k] > 0.0f ? vv[k] : 0.0f;
        c = c < lim[k] ? c : lim[k];
        o.rect[k] = (int)c;
    }
    if (o.rect[0] >= o.rect[2] || o.rect[1] >= o.rect[3]) return o;

    o.l11 = f_sqrt(f_div(cc, det));
    o.l21 = -f_div(cb, f_sqrt(f_mul(cc, det)));
    o.l22 = f_div(1.0f, f_sqrt(cc));
    o.mx = mx;
    o.my = my;
    o.visible = true;
    return o;
}

__device__ __forceinline__ void camera_centre(const DevCamera &cam, float (&c)[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
        c[j] = -(cam.R[j] * cam.t[0] + cam.R[3 + j] * cam.t[1] + cam.R[6 + j] * cam.t[2]);
}

// kTC: the MLP runs on tcgen05 (TMEM accumulators, one CTA = 128 rows);
// otherwise on mma.sync (one warp = 32 rows).
// kWide: the paper-width MLP (three hidden layers) on tcgen05, 128 rows per CTA.
template <bool kFP16, bool kMLP, bool kResidual, bool kTC, bool kWide = false>
__global__ void __launch_bounds__(kWide ? tcw::kThreads : (kTC ? tc::kThreads : kThreads))
    k_preprocess(RenderArgs args) {
    constexpr int kStep =
        kWide ? tcw::kThreads : (kTC ? tc::kThreads : kThreads);   // Gaussians per CTA step
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smem_raw);
    tc::Smem &tsm = *reinterpret_cast<tc::Smem *>(smem_raw);
    const DevCamera &cam = args.cam;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool tc = args.wt16 != nullptr && tc_raster(args);
    uint32_t tc_phase = 0;
    bool tc_ok = true;
    WideLayout wl{};
    if constexpr (kWide) {
        wl = wide_layout(args.mlp.h1, args.mlp.h2, args.mlp.h3);
        tcw::setup(smem_raw, wl, args.mlp);
    } else if constexpr (kMLP && kTC) {
        tc::setup(tsm, args.mlp);
    } else if constexpr (kMLP) {
        mlp_load_weights(sm, args.mlp);
        __syncthreads();
    }
    float cc[3];
    camera_centre(cam, cc);
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    float wbound = 0.0f;
    bool any_wide = false;
    unsigned nvis = 0;

    for (int64_t base = (int64_t)blockIdx.x * kStep; base < args.n;
         base += (int64_t)gridDim.x * kStep) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < args.n;
        float v[kRec];
        float qw = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
        bool qok = false;
        float P[3] = {0.f, 0.f, 0.f};
        if (valid) {
            load_record<kFP16>(args.attrs, i, v);
            qok = contract_quat(v, qw, qx, qy, qz);
            float d0 = v[0] - cc[0], d1 = v[1] - cc[1], d2 = v[2] - cc[2];
            float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            P[0] = d0 * inv;
            P[1] = d1 * inv;
            P[2] = d2 * inv;
        }
        float phi = 1.0f, opa = 0.f, dres[3] = {0.f, 0.f, 0.f};
        if constexpr (kMLP) {
            // feature row [P, s, q_hat, Y]
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
            float o[5];
            if constexpr (kWide) {
                tcw::put_features(smem_raw, wl, f);
                tc_ok &= tcw::mlp_cta(smem_raw, wl, args.mlp.h1, args.mlp.h2, args.mlp.h3,
                                      tc_phase, o);
            } else if constexpr (kTC) {
                tc::put_features(tsm, f);
                tc_ok &= tc::mlp_cta(tsm, tc_phase, o);
            } else {
                // BF16 row in shared memory (row = lane), one warp per 32 rows
                __nv_bfloat16 *xr = &sm.x[warp][lane * kXStride];
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
                mlp_warp<false>(sm, warp, lane, nullptr, nullptr);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 5; ++k) o[k] = sm.out[warp][lane][k];
                __syncwarp();
            }
            phi = fmaxf(o[0], 0.f);
            opa = 1.0f / (1.0f + __expf(-o[1]));
            dres[0] = o[2];
            dres[1] = o[3];
            dres[2] = o[4];
        }
        if (!valid) continue;
        if constexpr (!kMLP) opa = v[10];

        Contract c = contract_project(v, qw, qx, qy, qz, qok, cam);
        if (!c.visible) {
            args.rect[i] = make_uint2(0u, 0u);
            continue;
        }
        // degree-1 SH colour (Sec. 3.2), 3DGS basis signs
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float col = C0 * v[11 + ch] - C1 * P[1] * v[14 + ch] + C1 * P[2] * v[17 + ch] -
                        C1 * P[0] * v[20 + ch] + 0.5f;
            if constexpr (kResidual) col += dres[ch];
            rgb[ch] = fmaxf(col, 0.f);
        }
        // Eq. 3
        const float d = c.tz;
        const float smax = fmaxf(fmaxf(v[3], v[4]), v[5]);
        const float rz = 1.0f / d;
        const float w = phi * phi + phi * rz * rz + expf(smax * rz);
        ProjRec r;
        r.a = make_float4(c.mx, c.my, c.l11, c.l21);
        r.b = make_float4(c.l22, __log2f(opa), -w, -w * rgb[0]);
        r.c = make_float4(-w * rgb[1], -w * rgb[2], c.tz, -w * c.tz);
        args.rec[i] = r;
        if (kFP16 && tc) args.wt16[i] = weights_f16(r, 1.0f);   // rescaled by binning if needed
        // weights outside the range of the FP16 tensor-core sums
        const float wm = w * fmaxf(fmaxf(1.0f, rgb[0]), fmaxf(rgb[1], rgb[2]));
        const bool wide = !(w >= 1.0f && wm < kWideWeight);
        args.rect[i] = make_uint2((unsigned)c.rect[0] | ((unsigned)c.rect[2] << 16),
                                  (unsigned)c.rect[1] | ((unsigned)c.rect[3] << 16) |
                                      (wide ? kRectWide : 0u));
        if (wide) any_wide = true;
        else wbound = fmaxf(wbound, wm);
        ++nvis;
    }
    // bound on the rasteriser's weights |w|, |w c| for this frame (Gaussians
    // that are not wide)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wbound = fmaxf(wbound, __shfl_xor_sync(0xffffffffu, wbound, o));
    if ((threadIdx.x & 31) == 0 && wbound > 0.0f)
        atomicMax(&args.status->wmax_bits, __float_as_uint(wbound));
    if (__any_sync(0xffffffffu, any_wide) && (threadIdx.x & 31) == 0)
        atomicOr(&args.status->wide_bits, 1u);
    nvis = __reduce_add_sync(0xffffffffu, nvis);
    if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(&args.status->visible, nvis);
    if constexpr (kWide) {
        tcw::teardown(smem_raw, wl);
        if (!tc_ok && threadIdx.x == 0) atomicOr(&args.status->overflow, kStatusMmaTimeout);
    } else if constexpr (kMLP && kTC) {
        tc::teardown(tsm);
        if (!tc_ok && threadIdx.x == 0) atomicOr(&args.status->overflow, kStatusMmaTimeout);
    }
}

template <bool kFP16, bool kResidual>
cudaError_t launch_wide(const RenderArgs &a, int sm_count, cudaStream_t stream) {
    const size_t smem = wide_mlp_smem(a.mlp.h1, a.mlp.h2, a.mlp.h3);
    auto kern = k_preprocess<kFP16, true, kResidual, true, true>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one CTA per SM (shared memory), each holding 256 TMEM columns
    int64_t blocks = (a.n + tcw::kThreads - 1) / tcw::kThreads;
    if (blocks > sm_count) blocks = sm_count;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, tcw::kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <bool kFP16, bool kMLP, bool kResidual, bool kTC>
cudaError_t launch_t(const RenderArgs &a, int sm_count, cudaStream_t stream) {
    const size_t smem = kMLP ? (kTC ? sizeof(tc::Smem) : sizeof(MlpSmem)) : 16;
    auto kern = k_preprocess<kFP16, kMLP, kResidual, kTC>;
    if (kMLP) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = (kMLP && kTC) ? tc::kThreads : kThreads;
    int64_t blocks = (a.n + threads - 1) / threads;
    // tcgen05: at most 3 CTAs per SM (shared memory; 3 x 128 of the SM's 512
    // TMEM columns)
    const int64_t cap = (int64_t)sm_count * ((kMLP && kTC) ? 3 : 8);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, threads, smem, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_preprocess(const RenderArgs &a, int sm_count, cudaStream_t stream) {
    const bool fp16 = a.precision == MGS_PREC_FP16;
    const bool sync_mma = (a.flags & MGS_FLAG_MLP_MMA_SYNC) != 0;
    if (a.use_mlp && a.mlp.h1 != 0) {
        if (a.rgb_residual)
            return fp16 ? launch_wide<true, true>(a, sm_count, stream)
                        : launch_wide<false, true>(a, sm_count, stream);
        return fp16 ? launch_wide<true, false>(a, sm_count, stream)
                    : launch_wide<false, false>(a, sm_count, stream);
    }
    if (a.use_mlp) {
        if (sync_mma) {
            if (a.rgb_residual)
                return fp16 ? launch_t<true, true, true, false>(a, sm_count, stream)
                            : launch_t<false, true, true, false>(a, sm_count, stream);
            return fp16 ? launch_t<true, true, false, false>(a, sm_count, stream)
                        : launch_t<false, true, false, false>(a, sm_count, stream);
        }
        if (a.rgb_residual)
            return fp16 ? launch_t<true, true, true, true>(a, sm_count, stream)
                        : launch_t<false, true, true, true>(a, sm_count, stream);
        return fp16 ? launch_t<true, true, false, true>(a, sm_count, stream)
                    : launch_t<false, true, false, true>(a, sm_count, stream);
    }
    return fp16 ? launch_t<true, false, false, false>(a, sm_count, stream)
                : launch_t<false, false, false, false>(a, sm_count, stream);
}

}  // namespace mgs
