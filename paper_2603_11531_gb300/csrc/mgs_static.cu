// Allocation-free render entry point (mgs_render_static).
//
// Some callers cannot call cudaMalloc at render time: code running where the
// device allocator is forbidden or unavailable (for example inside a host
// callback, a plugin whose host application owns all device memory, or a
// real-time loop that must not take the allocator's locks or fail on an
// out-of-memory condition).  This entry point serves them: every byte of
// scratch it needs lives in one file-scope __device__ array of fixed size,
// which each GPU that loads this library holds until the process exits.
//
// Limits: at most kMaxGaussians Gaussians, kMaxTiles 16x16 tiles (e.g. up to
// 1920x1080), kMaxPairs (tile, Gaussian) intersections, plain mode (phi = 1,
// stored opacity; no enhancement MLP).  All calls share the one array, so
// calls whose GPU work overlaps (other streams, other host threads) race and
// corrupt each other's results; order them on one stream or serialise them.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mgs_internal.cuh"

namespace {

using namespace mgs;

constexpr int64_t kMaxGaussians = 131072;
constexpr int kMaxTiles = 8192;
constexpr int64_t kMaxPairs = int64_t(1) << 22;
constexpr int kMaxBinCtas = (int)((kMaxGaussians + 1023) / 1024);  // bin_ctas() bound

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kRecOff = 0;
constexpr size_t kRectOff = kRecOff + align256(kMaxGaussians * sizeof(ProjRec));
constexpr size_t kCountOff = kRectOff + align256(kMaxGaussians * sizeof(uint2));
constexpr size_t kOffsetsOff = kCountOff + align256((kMaxTiles + 1) * sizeof(uint32_t));
constexpr size_t kOrderOff = kOffsetsOff + align256((kMaxTiles + 1) * sizeof(uint32_t));
constexpr size_t kBasesOff = kOrderOff + align256((kMaxTiles + 1) * sizeof(uint32_t));
constexpr size_t kGidsOff =
    kBasesOff + align256((size_t)bin_scratch_words_for(kMaxBinCtas, kMaxTiles, kMaxGaussians) * sizeof(uint32_t));
constexpr size_t kWt16Off = kGidsOff + align256(kMaxPairs * sizeof(uint32_t));
constexpr size_t kStatusOff = kWt16Off + align256(kMaxGaussians * sizeof(uint4));
constexpr size_t kScratchBytes = kStatusOff + align256(sizeof(DevStatus));  // 30,557,440 B
static_assert(kScratchBytes == 30557440, "the documented size of the static scratch");

// The scratch.  In host code this name is only a host-side stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

mgs_status fail_static(mgs_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

// Once per device, with that device current: the array's device address and
// the SM count (used to size the launches).
mgs_status setup(int dev, unsigned char **scratch, int *sm_count) {
    if (dev < 0 || dev >= kMaxDevices)
        return fail_static(MGS_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail_static(MGS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        int sm = 0;
        e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sm <= 0)
            return fail_static(MGS_ERR_CUDA, "cannot query the SM count");
        g_sm_count[dev] = sm;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *scratch = g_scratch_dev[dev];
    *sm_count = g_sm_count[dev];
    return MGS_OK;
}

}  // namespace

extern "C" mgs_status mgs_render_static(const void *attrs, int64_t n, int32_t precision,
                                        const mgs_camera *cam, const mgs_render_opts *opts,
                                        float *out_rgb, mgs_stream stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (n < 0 || n > kMaxGaussians)
        return fail_static(MGS_ERR_INVALID_ARG, "n outside 0..131072 (allocation-free limit)");
    if (precision != MGS_PREC_FP32 && precision != MGS_PREC_FP16)
        return fail_static(MGS_ERR_INVALID_ARG, "unknown precision");
    if (n > 0 && (!attrs || (reinterpret_cast<uintptr_t>(attrs) & 15)))
        return fail_static(MGS_ERR_INVALID_ARG, "attrs must be a 16-byte aligned device pointer");
    if (!cam || !opts || !out_rgb) return fail_static(MGS_ERR_INVALID_ARG, "NULL argument");
    if (validate_camera(cam) != MGS_OK) return MGS_ERR_INVALID_ARG;
    const int tiles_x = (cam->width + kTile - 1) / kTile;
    const int tiles_y = (cam->height + kTile - 1) / kTile;
    if ((int64_t)tiles_x * tiles_y > kMaxTiles)
        return fail_static(MGS_ERR_INVALID_ARG, "image needs more than 8192 tiles (allocation-free limit)");
    if (opts->use_mlp)
        return fail_static(MGS_ERR_INVALID_ARG, "the allocation-free entry point renders without the MLP");
    // Only flags this entry point honours: the sorted comparator and the MLP
    // options would silently render something other than what was asked for.
    if (opts->flags & ~(uint32_t)(MGS_FLAG_NO_CULL | MGS_FLAG_RASTER_FMA))
        return fail_static(MGS_ERR_INVALID_ARG,
                           "the allocation-free entry point accepts only MGS_FLAG_NO_CULL and "
                           "MGS_FLAG_RASTER_FMA");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail_static(MGS_ERR_CUDA, "cudaGetDevice failed");
    unsigned char *S = nullptr;
    int sm_count = 0;
    mgs_status st = setup(dev, &S, &sm_count);
    if (st != MGS_OK) return st;

    RenderArgs a{};
    a.attrs = attrs;
    a.n = n;
    a.precision = precision;
    memcpy(a.cam.R, cam->R, sizeof a.cam.R);
    memcpy(a.cam.t, cam->t, sizeof a.cam.t);
    a.cam.fx = cam->fx;
    a.cam.fy = cam->fy;
    a.cam.cx = cam->cx;
    a.cam.cy = cam->cy;
    a.cam.width = cam->width;
    a.cam.height = cam->height;
    a.cam.znear = cam->znear;
    a.cam.tiles_x = tiles_x;
    a.cam.tiles_y = tiles_y;
    a.bg[0] = opts->bg[0];
    a.bg[1] = opts->bg[1];
    a.bg[2] = opts->bg[2];
    a.flags = opts->flags;
    a.rec = reinterpret_cast<ProjRec *>(S + kRecOff);
    a.rect = reinterpret_cast<uint2 *>(S + kRectOff);
    a.tile_count = reinterpret_cast<uint32_t *>(S + kCountOff);
    a.tile_offsets = reinterpret_cast<uint32_t *>(S + kOffsetsOff);
    a.tile_order = reinterpret_cast<uint32_t *>(S + kOrderOff);
    a.gids = reinterpret_cast<uint32_t *>(S + kGidsOff);
    a.wt16 = reinterpret_cast<uint4 *>(S + kWt16Off);
    a.capacity = (uint64_t)kMaxPairs;
    a.status = reinterpret_cast<DevStatus *>(S + kStatusOff);
    a.out_rgb = out_rgb;
    uint32_t *bases = reinterpret_cast<uint32_t *>(S + kBasesOff);

    // the array keeps the previous call's contents: clear what starts at zero
    // (tile counts are cleared by the binning launch itself)
    cudaError_t e = cudaMemsetAsync(a.status, 0, sizeof(DevStatus), stream);
    if (e == cudaSuccess && n > 0) e = launch_preprocess(a, sm_count, stream);
    if (e == cudaSuccess) e = launch_binning(a, sm_count, bases, stream);
    if (e == cudaSuccess) e = launch_raster(a, stream);
    DevStatus h{};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, a.status, sizeof h, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    char msg[160];
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "CUDA error: %s", cudaGetErrorString(e));
        return fail_static(MGS_ERR_CUDA, msg);
    }
    if (h.overflow & kStatusMmaTimeout)
        return fail_static(MGS_ERR_TIMEOUT, "a tensor-core MMA wait in preprocessing timed out");
    if (h.last_pairs > (unsigned long long)kMaxPairs) {
        snprintf(msg, sizeof msg,
                 "view needs %llu (tile, Gaussian) pairs; the allocation-free limit is %lld",
                 (unsigned long long)h.last_pairs, (long long)kMaxPairs);
        return fail_static(MGS_ERR_OVERFLOW, msg);
    }
    return MGS_OK;
}
