// Internal declarations shared by the CUDA translation units of the renderer.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mobilegs.h"

namespace mgs {

constexpr int kTile = 16;         // tile edge in pixels (binning granularity)
constexpr int kRec = 24;          // stored elements per Gaussian
constexpr int kMlpIn = 22;        // [P(3), s(3), q(4), Y(12)]
constexpr int kMlpK1 = 32;        // layer-1 K padded for the MMA
constexpr int kMlpHidden = 64;
constexpr int kMlpOut = 5;        // phi, o, d_r, d_g, d_b
constexpr int kMlpN3 = 8;         // head N padded for the MMA

// Camera as the kernels see it.
struct DevCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int width, height;
    float znear;
    int tiles_x, tiles_y;
};

// Packed MLP weights in device memory (BF16, row-major [out][in], padded).
struct DevMLP {
    const __nv_bfloat16 *w1;  // [64][32]        wide: [h1][32]
    const __nv_bfloat16 *w2;  // [64][64]        wide: [h2][h1]
    const __nv_bfloat16 *w3;  // [8][64] (head)  wide: [h3][h2]
    const float *b1;          // [64]            wide: [h1]
    const float *b2;          // [64]            wide: [h2]
    const float *b3;          // [8]             wide: [h3]
    const __nv_bfloat16 *w4;  // wide only: head [8][h3]
    const float *b4;          // wide only: [8]
    int h1, h2, h3;           // 0: the 22-64-64-5 MLP; else App. C's three hidden layers
};

// Shared-memory layout (byte offsets) of the wide (three hidden layer)
// tcgen05 MLP, two 128-row tiles per step: BF16 operands in canonical K-major
// layout (features x of both tiles, activations a0/a1 of the current tile,
// weights w1..w3), the FP32 head ([h3][8], input-major, outputs 5..7 zero),
// biases, and the head partial sums exchanged between the two warp halves.
struct WideLayout {
    uint32_t x, a0, a1, w1, w2, w3, head, b1, b2, b3, b4, red, mbar, tmem, total;
};
__host__ __device__ inline WideLayout wide_layout(int h1, int h2, int h3) {
    WideLayout L{};
    uint32_t o = 0;
    auto take = [&o](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) / align * align;
        const uint32_t r = o;
        o += bytes;
        return r;
    };
    L.x = take(2u * 128u * 32u * 2u, 128u);   // features of the step's two tiles
    L.a0 = take(128u * (uint32_t)h1 * 2u, 128u);
    L.a1 = take(128u * (uint32_t)h2 * 2u, 128u);
    L.w1 = take((uint32_t)h1 * 32u * 2u, 128u);
    L.w2 = take((uint32_t)h2 * (uint32_t)h1 * 2u, 128u);
    L.w3 = take((uint32_t)h3 * (uint32_t)h2 * 2u, 128u);
    L.head = take(8u * (uint32_t)h3 * 4u, 16u);
    L.b1 = take((uint32_t)h1 * 4u, 16u);
    L.b2 = take((uint32_t)h2 * 4u, 16u);
    L.b3 = take((uint32_t)h3 * 4u, 16u);
    L.b4 = take(8u * 4u, 16u);
    L.red = take(128u * 8u * 4u, 16u);        // head partial sums of one warp half
    L.mbar = take(8u, 8u);
    L.tmem = take(4u, 4u);
    L.total = o;
    return L;
}
inline size_t wide_mlp_smem(int h1, int h2, int h3) { return wide_layout(h1, h2, h3).total; }

// Device-visible status of a workspace (accumulates until the host syncs).
constexpr unsigned kStatusOverflow = 1u;    // some render exceeded its pair capacity
constexpr unsigned kStatusMmaTimeout = 2u;  // a tcgen05 MMA wait ran out (results invalid)
struct DevStatus {
    unsigned int overflow;          // kStatus* bits seen since the last sync
    // Nonzero when the current frame has a Gaussian whose weight the FP16
    // tensor-core sums cannot hold next to the others (kRectWide): set by
    // preprocessing, read by the count kernel of binning, reset by
    // k_scan_order.
    unsigned int wide_bits;
    unsigned long long max_pairs;   // largest pair count seen since the last sync
    unsigned long long last_pairs;  // pair count of the most recent render
    // Largest |w c| and w over the visible Gaussians (FP32 bits; positive
    // floats order as unsigned integers): accumulated by preprocessing,
    // handed to the frame's rasteriser (wmax_frame_bits) and reset by
    // k_scan_order, which runs between the two.
    unsigned int wmax_bits;
    unsigned int wmax_frame_bits;
    // Visible Gaussians (accumulated by preprocessing) and tiles marked
    // kTileWide; k_scan_order hands both to last_* and resets the first.
    unsigned int visible;
    unsigned int last_visible;
    unsigned int last_wide_tiles;
    unsigned int pad;
};

// Weight range of the tensor-core sums.  The rasteriser of FP16 scenes sums
// a w c and a w in FP16 x FP16 products scaled by one power of two per frame
// (largest weight into [2^14, 2^15)).  Eq. 3 gives w >= 1 for every Gaussian
// in front of the camera, so weights below kWideWeight keep at least 2^-5
// after scaling, and their FP16 high + low parts at least 20 bits.  A
// Gaussian with w * max(1, c) >= kWideWeight (or w < 1, or not finite) is
// "wide": preprocessing sets kRectWide in its rectangle, binning marks every
// tile that lists it (kTileWide in the tile's rasterisation-order entry), and
// those tiles take the FP32 FMA sums instead.  The frame's scale is taken
// over the other Gaussians only.
constexpr float kWideWeight = 1048576.0f;   // 2^20
constexpr unsigned kRectWide = 0x80000000u; // in rect.y (above y_hi << 16)
constexpr unsigned kTileWide = 0x80000000u; // in tile_order[] and tile_count[]
constexpr unsigned kTileMask = 0x7FFFFFFFu;

// Projected Gaussian (48 bytes), written by preprocessing, read by the
// rasteriser:
//   a = (m_x, m_y, l11, l21)          FP32-contract mean and factors
//   b = (l22, log2 o, -w, -w c_r)
//   c = (-w c_g, -w c_b, view depth d (FP32 contract), -w d)
// The inclusion test is q = (l11 dx + l21 dy)^2 + (l22 dy)^2 <= 9 with
// dx = x + 0.5 - m_x, dy = y + 0.5 - m_y, evaluated exactly as
// e1 = fma(l11, dx, l21*dy), e2 = l22*dy, q = fma(e1, e1, e2*e2).
struct __align__(16) ProjRec {
    float4 a, b, c;
};

struct RenderArgs {
    const void *attrs;
    int64_t n;
    int precision;
    int use_mlp;
    int rgb_residual;
    DevMLP mlp;
    DevCamera cam;
    float bg[3];
    unsigned flags;
    // workspace
    ProjRec *rec;
    uint2 *rect;              // packed (x_lo | x_hi << 16, y_lo | y_hi << 16 | kRectWide)
    uint32_t *tile_count;     // [T]
    uint32_t *tile_offsets;   // [T + 1]
    uint32_t *tile_order;     // [T] rasterisation order (longest lists first), | kTileWide
    uint32_t *gids;           // [capacity]
    uint4 *wt16;              // [n] tensor-core weights (FP16 high / low parts), see tc_raster()
    const uint32_t *perm;     // [n] stored position -> caller index (null: identity)
    const uint32_t *iperm;    // [n] caller index -> stored position (null: identity)
    uint64_t capacity;
    DevStatus *status;
    // outputs
    float *out_rgb;
    float *out_aux;
    int32_t *out_count;
    float *out_depth;          // depth image (Eq. 5), optional
};

// Does this render rasterise with tensor-core sums (FP16 attributes, no
// comparator, not forced onto the FMA pipe)?  Preprocessing then also writes
// every visible Gaussian's weights in FP16 (args.wt16; binning rescales them
// when the frame's largest weight needs it).  A depth image
// rendered this way takes its numerator sum d a w in FP32 and its
// denominator from the tensor-core B.
__host__ __device__ inline bool tc_raster(const RenderArgs &a) {
    return a.precision == MGS_PREC_FP16 &&
           (a.flags & (MGS_FLAG_RASTER_FMA | MGS_FLAG_SORTED)) == 0;
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

// Can Gaussian (m, l) include any pixel centre of the block centred at (bx, by)
// with half extents (hx, hy)?  In the whitened coordinates e1 = l11 dx +
// l21 dy, e2 = l22 dy an included pixel lies in the disc e1^2 + e2^2 <= 9, so
// inside the octagon |e1|, |e2| <= 3 and |e1 +- e2| <= 3 sqrt(2); the block
// maps to a parallelogram, and each of the four slab tests compares the
// block centre's coordinate with the parallelogram's half extent along it.
// Sound for the exact FP32 test: the margin (2^-18 relative, twice that for
// the diagonal slabs) covers the rounding of the test and of the FP32
// predicate.  The diagonal slabs remove about 14% of the (block, Gaussian)
// candidates that the axis slabs alone keep.
__device__ __forceinline__ bool block_may_hit(float mx, float my, float l11, float l21, float l22,
                                              float bx, float by, float hx, float hy) {
    const float dxb = bx - mx, dyb = by - my;
    const float e1 = fmaf(l11, dxb, l21 * dyb);
    const float e2 = l22 * dyb;
    const float a11 = fabsf(l11), a21 = fabsf(l21), a22 = fabsf(l22);
    const float m = 3.814697265625e-06f *
                    fmaf(a11, fabsf(dxb) + hx, fmaf(a21 + a22, fabsf(dyb) + hy, 4.0f));
    const float xh = a11 * hx;
    const float h1 = fmaf(a21, hy, xh);
    const float h2 = a22 * hy;
    const float hu = fmaf(fabsf(l21 + l22), hy, xh);
    const float hv = fmaf(fabsf(l21 - l22), hy, xh);
    const float r2 = 4.2426410f + 2.0f * m;   // 3 sqrt(2), rounded up
    return (fabsf(e1) - h1 <= 3.0f + m) && (fabsf(e2) - h2 <= 3.0f + m) &&
           (fabsf(e1 + e2) - hu <= r2) && (fabsf(e1 - e2) - hv <= r2);
}

// Scratch of the sorted comparator (mgs_sorted.cu).
struct SortedScratch {
    uint32_t *nkeys, *nkeys_tmp;   // [n]   depth ranking: FP32-contract depth bits
    uint32_t *nvals, *nvals_tmp;   // [n]
    uint32_t *rank;                // [n]
    uint32_t *keys, *keys_tmp;     // [capacity] rank of each list entry
    uint32_t *vals, *vals_tmp;     // [capacity]
    void *temp;                    // library sort temporary storage
    size_t temp_bytes;
};
// Temporary storage the comparator's sorts need for n Gaussians, `capacity`
// list entries and T tiles.
size_t sorted_temp_bytes(int64_t n, int64_t capacity, int T);
int64_t sorted_hist_entries(int64_t n_max);
// Stable LSD radix sort of (key, value) pairs by key bits [begin_bit, end_bit).
cudaError_t radix_sort(uint64_t **k, uint32_t **v, uint64_t **kt, uint32_t **vt, int64_t n_max,
                       const unsigned long long *n_dev, int begin_bit, int end_bit,
                       uint32_t *hist, cudaStream_t stream);
// Load-time spatial order (mgs_order.cu): attrs_out = attrs_in sorted along a
// Morton curve of the means; perm[j] = caller index of stored row j, iperm
// its inverse.  Synchronous.
cudaError_t spatial_order(const void *attrs_in, int64_t n, int precision, void *attrs_out,
                          uint32_t *perm, uint32_t *iperm, cudaStream_t stream);
// out[j] = perm[in[j]] for j < count.
cudaError_t map_ids(const uint32_t *in, const uint32_t *perm, int64_t count, uint32_t *out,
                    cudaStream_t stream);
// Depth-sorts every tile list and blends front to back (Eq. 11 comparator).
cudaError_t launch_sorted(const RenderArgs &a, const SortedScratch &s, cudaStream_t stream);

// Launchers (each enqueues its kernels on `stream`).
cudaError_t launch_preprocess(const RenderArgs &a, int sm_count, cudaStream_t stream);
// Per-tile counts, scan and scatter.  `scratch` has bin_scratch_words(n, T,
// sm_count) 32-bit words: the per-CTA tile bases, then the pair counts of the
// 32-Gaussian groups and their exclusive scan.
// marks (nullable): three events recorded on `stream` after the plan (count
// reset, group pairs, plan scan), after the count and after the tile scan.
cudaError_t launch_binning(const RenderArgs &a, int sm_count, uint32_t *scratch, cudaStream_t stream,
                           const cudaEvent_t *marks = nullptr);
int bin_ctas(int64_t n, int sm_count);
__host__ __device__ constexpr int64_t bin_scratch_words_for(int64_t ctas, int64_t T, int64_t n) {
    return (ctas * T + 1) / 2 * 2 + 2 * ((n + 31) / 32 + 1) + (n + 31) / 32;
}
int64_t bin_scratch_words(int64_t n, int64_t T, int sm_count);
// Backward pass (mgs_backward.cu): gG [n][grad_record_size()] scratch,
// partials [pre_bwd_blocks()][mlp_grad_size()] scratch, d_attrs [n][24],
// d_mlp [mlp_grad_size()] (nullable).
cudaError_t launch_backward(const RenderArgs &a, int sm_count, const float *dL_drgb,
                            const float *aux, float *gG, float *d_attrs, float *d_mlp,
                            float *partials, cudaStream_t stream);
int mlp_grad_size();
int grad_record_size();
int pre_bwd_blocks(int64_t n, int sm_count);
// Sets the calling thread's message returned by mgs_last_error().
void set_last_error(const char *msg);
// Host-side camera check shared by every entry point: image size 1..16384,
// finite pose and intrinsics, focal lengths > 0, 0 < znear (finite).  Sets the
// error message on failure.
mgs_status validate_camera(const mgs_camera *c);
// Preprocessing and binning of one view into workspace w (no rasterisation,
// no allocation if the workspace is large enough); *args_out receives the
// arguments the rasteriser needs.  Stream-ordered, capturable.  args_only:
// check the arguments, size the workspace and fill *args_out, launch nothing.
mgs_status prepare_view(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                        const mgs_render_opts *opts, float *out_rgb, cudaStream_t stream,
                        RenderArgs *args_out, bool args_only = false);
// Changes whenever one of the workspace's scratch buffers is reallocated
// (launches captured before then address freed memory).
uint64_t workspace_generation(mgs_workspace w);
int ctx_device(mgs_ctx c);
int ctx_sm_count(mgs_ctx c);
int64_t scene_size(mgs_scene s);
mgs_ctx scene_ctx(mgs_scene s);
cudaError_t launch_raster(const RenderArgs &a, cudaStream_t stream);
// Persistent rasteriser over the tiles of `nviews` views (views_dev and
// prefix_dev in device memory; prefix has nviews + 1 entries).
cudaError_t launch_raster_batch(const RenderArgs *views_dev, const int *prefix_dev, int nviews,
                                unsigned *counter_dev, int sm_count, cudaStream_t stream);

}  // namespace mgs
