// Host side of the C-ABI declared in include/mobilegs.h: argument checks,
// device memory of scenes and workspaces, and the launch sequence of a render
// (preprocess -> scan -> scatter -> rasterise).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <array>
#include <vector>

#include "mgs_internal.cuh"

using namespace mgs;

namespace {

thread_local std::string g_err;

mgs_status fail(mgs_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

mgs_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(MGS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(MGS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

template <class T>
void dev_free(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

}  // namespace

struct mgs_ctx_s {
    int device = 0;
    int sm_count = 0;
};

struct mgs_scene_s {
    mgs_ctx ctx = nullptr;
    int64_t n = 0;
    int precision = MGS_PREC_FP32;
    void *attrs = nullptr;
    bool has_mlp = false;
    unsigned char *mlp_blob = nullptr;  // packed weights + biases
    DevMLP mlp{};
    uint32_t *perm = nullptr;    // stored row -> caller index (spatial order)
    uint32_t *iperm = nullptr;   // caller index -> stored row
    int64_t bytes = 0;
};

// Events per timed render: start, after preprocessing, after the binning plan,
// after the count, after the tile scan, after the scatter, after the raster.
constexpr int kStageEvents = 7;

struct mgs_workspace_s {
    mgs_ctx ctx = nullptr;
    int64_t n_cap = 0;
    int64_t tiles_cap = 0;
    uint64_t pair_cap = 0;
    int64_t img_cap = 0;
    ProjRec *rec = nullptr;
    uint4 *wt16 = nullptr;
    uint2 *rect = nullptr;
    uint32_t *tile_count = nullptr;
    uint32_t *tile_offsets = nullptr;
    uint32_t *tile_order = nullptr;
    uint32_t *gids = nullptr;
    uint32_t *bases = nullptr;   // binning scratch: [binning CTAs][tiles] block bases, group scan
    int64_t bases_cap = 0;
    float *img = nullptr;
    float *bwd_g = nullptr;        // backward: per-Gaussian raster gradients
    int64_t bwd_g_cap = 0;
    float *bwd_partials = nullptr; // backward: per-CTA MLP weight gradients
    int64_t bwd_partials_cap = 0;
    SortedScratch ss{};            // sorted comparator scratch
    int64_t ss_n_cap = 0, ss_pairs_cap = 0, ss_tiles_cap = 0;
    DevStatus *status = nullptr;
    int64_t last_tiles = 0;
    const uint32_t *last_perm = nullptr;   // storage -> caller order of the last scene
    uint64_t grow_hint = 0;  // pairs needed by an overflowed render
    uint64_t generation = 0; // bumped whenever a scratch buffer is reallocated
    bool timing = false;
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::array<cudaEvent_t, kStageEvents>> pending;  // per timed render
};

namespace {

int64_t ws_bytes(const mgs_workspace_s *w) {
    return w->n_cap * (int64_t)(sizeof(ProjRec) + sizeof(uint2) + sizeof(uint4)) +
           w->tiles_cap * 3 * (int64_t)sizeof(uint32_t) + (int64_t)w->pair_cap * 4 +
           w->img_cap * 12 + w->bases_cap * 4 + (int64_t)sizeof(DevStatus);
}

mgs_status ws_ensure(mgs_workspace_s *w, int64_t n, int64_t tiles, uint64_t pairs) {
    cudaError_t e;
    const uint64_t gen0 = w->generation;
    struct Bump {   // any reallocation below invalidates captured launches
        mgs_workspace_s *w;
        uint64_t gen0;
        const void *p[7];
        int64_t c[4];
        ~Bump() {
            const void *q[7] = {w->rec, w->rect, w->wt16, w->tile_count, w->gids, w->bases, w->status};
            const int64_t d[4] = {w->n_cap, w->tiles_cap, (int64_t)w->pair_cap, w->bases_cap};
            bool changed = false;
            for (int k = 0; k < 7; ++k) changed |= q[k] != p[k];
            for (int k = 0; k < 4; ++k) changed |= d[k] != c[k];
            if (changed) w->generation = gen0 + 1;
        }
    } bump{w, gen0, {w->rec, w->rect, w->wt16, w->tile_count, w->gids, w->bases, w->status},
           {w->n_cap, w->tiles_cap, (int64_t)w->pair_cap, w->bases_cap}};
    if (n > w->n_cap) {
        dev_free(w->rec);
        dev_free(w->rect);
        dev_free(w->wt16);
        w->n_cap = 0;
        if ((e = dev_alloc(&w->rec, (size_t)n)) != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = dev_alloc(&w->rect, (size_t)n)) != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = dev_alloc(&w->wt16, (size_t)n)) != cudaSuccess) return cuda_fail(e, "workspace");
        w->n_cap = n;
    }
    if (tiles + 1 > w->tiles_cap) {
        dev_free(w->tile_count);
        dev_free(w->tile_offsets);
        dev_free(w->tile_order);
        w->tiles_cap = 0;
        const size_t t = (size_t)tiles + 1;
        if ((e = dev_alloc(&w->tile_count, t)) != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = dev_alloc(&w->tile_offsets, t)) != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = dev_alloc(&w->tile_order, t)) != cudaSuccess) return cuda_fail(e, "workspace");
        w->tiles_cap = (int64_t)t;
    }
    if (pairs > w->pair_cap) {
        if (pairs > 0xFFFFFFFFull) pairs = 0xFFFFFFFFull;
        dev_free(w->gids);
        w->pair_cap = 0;
        if ((e = dev_alloc(&w->gids, (size_t)pairs)) != cudaSuccess) return cuda_fail(e, "workspace");
        w->pair_cap = pairs;
    }
    const int64_t nb = bin_scratch_words(n, tiles, w->ctx->sm_count);
    if (nb > w->bases_cap) {
        dev_free(w->bases);
        w->bases_cap = 0;
        if ((e = dev_alloc(&w->bases, (size_t)nb)) != cudaSuccess) return cuda_fail(e, "workspace");
        w->bases_cap = nb;
    }
    if (!w->status) {
        if ((e = dev_alloc(&w->status, 1)) != cudaSuccess) return cuda_fail(e, "workspace");
        if ((e = cudaMemset(w->status, 0, sizeof(DevStatus))) != cudaSuccess)
            return cuda_fail(e, "workspace");
    }
    return MGS_OK;
}

mgs_status check_camera(const mgs_camera *c) {
    if (!c) return fail(MGS_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(MGS_ERR_INVALID_ARG, "image size %dx%d outside 1..16384", c->width, c->height);
    if (!finite_pos(c->fx) || !finite_pos(c->fy))
        return fail(MGS_ERR_INVALID_ARG, "focal lengths must be finite and > 0");
    if (!std::isfinite(c->cx) || !std::isfinite(c->cy))
        return fail(MGS_ERR_INVALID_ARG, "principal point must be finite");
    // the pinhole projection divides by the view depth: the near plane must
    // lie in front of the camera (this also keeps Eq. 3's depth d > 0)
    if (!finite_pos(c->znear)) return fail(MGS_ERR_INVALID_ARG, "znear must be finite and > 0");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(c->R[i])) return fail(MGS_ERR_INVALID_ARG, "R must be finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(c->t[i])) return fail(MGS_ERR_INVALID_ARG, "t must be finite");
    return MGS_OK;
}

DevCamera to_dev(const mgs_camera *c) {
    DevCamera d;
    memcpy(d.R, c->R, sizeof d.R);
    memcpy(d.t, c->t, sizeof d.t);
    d.fx = c->fx;
    d.fy = c->fy;
    d.cx = c->cx;
    d.cy = c->cy;
    d.width = c->width;
    d.height = c->height;
    d.znear = c->znear;
    d.tiles_x = (c->width + kTile - 1) / kTile;
    d.tiles_y = (c->height + kTile - 1) / kTile;
    return d;
}

uint64_t default_pairs(int64_t n) {
    uint64_t p = (uint64_t)n * 24u;
    return p < (1u << 20) ? (1u << 20) : p;
}

// Backward request: when non-null, render_impl builds the frame's records and
// tile lists and then runs the adjoint kernels instead of the rasteriser.
struct BackwardIO {
    const float *dL_drgb;
    const float *aux;
    float *d_attrs;
    float *d_mlp;
};

mgs_status render_impl(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                       const mgs_render_opts *opts, float *out_rgb, float *out_aux,
                       int32_t *out_count, cudaStream_t stream,
                       const BackwardIO *bwd = nullptr, RenderArgs *prep = nullptr,
                       float *out_depth = nullptr, bool args_only = false) {
    if (!w || !s) return fail(MGS_ERR_INVALID_ARG, "workspace or scene is NULL");
    if (w->ctx != s->ctx) return fail(MGS_ERR_INVALID_ARG, "scene and workspace belong to different contexts");
    mgs_status st = check_camera(cam);
    if (st != MGS_OK) return st;
    if (!opts) return fail(MGS_ERR_INVALID_ARG, "opts is NULL");
    if (!out_rgb && !bwd && !prep) return fail(MGS_ERR_INVALID_ARG, "out_rgb is NULL");
    if (opts->use_mlp && !s->has_mlp)
        return fail(MGS_ERR_INVALID_ARG, "use_mlp requested but the scene has no MLP weights");
    if (opts->use_mlp && s->mlp.h1 != 0) {
        if (opts->flags & MGS_FLAG_MLP_MMA_SYNC)
            return fail(MGS_ERR_INVALID_ARG, "the paper-width MLP runs on tcgen05 only");
        if (bwd) return fail(MGS_ERR_INVALID_ARG, "no backward pass for the paper-width MLP");
    }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(opts->bg[k])) return fail(MGS_ERR_INVALID_ARG, "bg must be finite");
    DeviceGuard g(w->ctx->device);
    if (!g.ok) return fail(MGS_ERR_CUDA, "cannot select device %d", w->ctx->device);

    const DevCamera dc = to_dev(cam);
    const int64_t T = (int64_t)dc.tiles_x * dc.tiles_y;
    uint64_t want = w->pair_cap ? w->pair_cap : default_pairs(s->n);
    if (w->grow_hint > want) want = w->grow_hint;
    st = ws_ensure(w, s->n, T, want);
    if (st != MGS_OK) return st;

    RenderArgs a{};
    a.attrs = s->attrs;
    a.n = s->n;
    a.precision = s->precision;
    a.use_mlp = opts->use_mlp ? 1 : 0;
    a.rgb_residual = (opts->use_mlp && opts->mlp_rgb_residual) ? 1 : 0;
    a.mlp = s->mlp;
    a.cam = dc;
    a.bg[0] = opts->bg[0];
    a.bg[1] = opts->bg[1];
    a.bg[2] = opts->bg[2];
    a.flags = opts->flags;
    a.rec = w->rec;
    a.rect = w->rect;
    a.wt16 = w->wt16;
    a.perm = s->perm;
    a.iperm = s->iperm;
    a.tile_count = w->tile_count;
    a.tile_offsets = w->tile_offsets;
    a.tile_order = w->tile_order;
    a.gids = w->gids;
    a.capacity = w->pair_cap;
    a.status = w->status;
    a.out_rgb = out_rgb;
    a.out_aux = out_aux;
    a.out_count = out_count;
    a.out_depth = out_depth;
    if (out_depth && (out_aux || out_count || (opts->flags & MGS_FLAG_SORTED)))
        return fail(MGS_ERR_INVALID_ARG, "the depth image is rendered without aux, counts or sorting");
    if (prep && args_only) {   // arguments of this view; nothing is launched
        *prep = a;
        return MGS_OK;
    }

    std::array<cudaEvent_t, kStageEvents> ev{};
    cudaError_t e = cudaSuccess;
    if (w->timing) {
        for (auto &x : ev) {
            if (w->event_pool.empty()) {
                if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "event");
            } else {
                x = w->event_pool.back();
                w->event_pool.pop_back();
            }
        }
        cudaEventRecord(ev[0], stream);
    }
    if (s->n > 0 && (e = launch_preprocess(a, w->ctx->sm_count, stream)) != cudaSuccess)
        return cuda_fail(e, "preprocess launch");
    if (w->timing) cudaEventRecord(ev[1], stream);
    if ((e = launch_binning(a, w->ctx->sm_count, w->bases, stream,
                            w->timing ? &ev[2] : nullptr)) != cudaSuccess)
        return cuda_fail(e, "binning launch");
    if (w->timing) cudaEventRecord(ev[5], stream);
    if (opts->flags & MGS_FLAG_SORTED) {
        if (out_aux) return fail(MGS_ERR_INVALID_ARG, "the sorted comparator has no aux output");
        const int64_t nc = s->n > 0 ? s->n : 1;
        const int64_t pc = (int64_t)w->pair_cap;
        if (nc > w->ss_n_cap || pc > w->ss_pairs_cap || T > w->ss_tiles_cap) {
            SortedScratch &q = w->ss;
            dev_free(q.nkeys); dev_free(q.nkeys_tmp); dev_free(q.nvals); dev_free(q.nvals_tmp);
            dev_free(q.rank); dev_free(q.keys); dev_free(q.keys_tmp); dev_free(q.vals);
            dev_free(q.vals_tmp);
            if (q.temp) cudaFree(q.temp);
            q.temp = nullptr;
            w->ss_n_cap = w->ss_pairs_cap = w->ss_tiles_cap = 0;
            q.temp_bytes = sorted_temp_bytes(nc, pc, (int)T);
            if ((e = dev_alloc(&q.nkeys, nc)) != cudaSuccess || (e = dev_alloc(&q.nkeys_tmp, nc)) != cudaSuccess ||
                (e = dev_alloc(&q.nvals, nc)) != cudaSuccess || (e = dev_alloc(&q.nvals_tmp, nc)) != cudaSuccess ||
                (e = dev_alloc(&q.rank, nc)) != cudaSuccess || (e = dev_alloc(&q.keys, pc)) != cudaSuccess ||
                (e = dev_alloc(&q.keys_tmp, pc)) != cudaSuccess || (e = dev_alloc(&q.vals, pc)) != cudaSuccess ||
                (e = dev_alloc(&q.vals_tmp, pc)) != cudaSuccess ||
                (e = cudaMalloc(&q.temp, q.temp_bytes ? q.temp_bytes : 16)) != cudaSuccess)
                return cuda_fail(e, "sorted scratch");
            w->ss_n_cap = nc;
            w->ss_pairs_cap = pc;
            w->ss_tiles_cap = T;
        }
        if ((e = launch_sorted(a, w->ss, stream)) != cudaSuccess) return cuda_fail(e, "sorted launch");
        if (w->timing) {
            cudaEventRecord(ev[6], stream);
            w->pending.push_back(ev);
        }
        w->last_tiles = T;
        w->last_perm = s->perm;
        return MGS_OK;
    }
    if (prep) {
        *prep = a;
        w->last_tiles = T;
        w->last_perm = s->perm;
        return MGS_OK;
    }
    if (bwd) {
        if (s->n > w->bwd_g_cap) {
            dev_free(w->bwd_g);
            w->bwd_g_cap = 0;
            if ((e = dev_alloc(&w->bwd_g, (size_t)s->n * grad_record_size())) != cudaSuccess)
                return cuda_fail(e, "workspace");
            w->bwd_g_cap = s->n;
        }
        const int64_t np = (int64_t)pre_bwd_blocks(s->n, w->ctx->sm_count) * mlp_grad_size();
        if (np > w->bwd_partials_cap) {
            dev_free(w->bwd_partials);
            w->bwd_partials_cap = 0;
            if ((e = dev_alloc(&w->bwd_partials, (size_t)np)) != cudaSuccess)
                return cuda_fail(e, "workspace");
            w->bwd_partials_cap = np;
        }
        if (s->n > 0 && (e = launch_backward(a, w->ctx->sm_count, bwd->dL_drgb, bwd->aux, w->bwd_g,
                                             bwd->d_attrs, bwd->d_mlp, w->bwd_partials,
                                             stream)) != cudaSuccess)
            return cuda_fail(e, "backward launch");
        if (s->n == 0 && bwd->d_mlp &&
            (e = cudaMemsetAsync(bwd->d_mlp, 0, (size_t)mlp_grad_size() * 4, stream)) != cudaSuccess)
            return cuda_fail(e, "memset");
    } else if ((e = launch_raster(a, stream)) != cudaSuccess) {
        return cuda_fail(e, "raster launch");
    }
    if (w->timing) {
        cudaEventRecord(ev[6], stream);
        w->pending.push_back(ev);
    }
    w->last_tiles = T;
    w->last_perm = s->perm;
    return MGS_OK;
}

}  // namespace

void mgs::set_last_error(const char *msg) { g_err = msg; }

mgs_status mgs::validate_camera(const mgs_camera *c) { return check_camera(c); }

mgs_status mgs::prepare_view(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                             const mgs_render_opts *opts, float *out_rgb, cudaStream_t stream,
                             RenderArgs *args_out, bool args_only) {
    mgs_status st = render_impl(w, s, cam, opts, out_rgb, nullptr, nullptr, stream, nullptr,
                                args_out, nullptr, args_only);
    if (st == MGS_OK) args_out->out_rgb = out_rgb;
    return st;
}

uint64_t mgs::workspace_generation(mgs_workspace w) { return w->generation; }

int mgs::ctx_device(mgs_ctx c) { return c->device; }
int mgs::ctx_sm_count(mgs_ctx c) { return c->sm_count; }
int64_t mgs::scene_size(mgs_scene s) { return s->n; }
mgs_ctx mgs::scene_ctx(mgs_scene s) { return s->ctx; }

extern "C" {

const char *mgs_last_error(void) { return g_err.c_str(); }
const char *mgs_version(void) { return "mobilegs-gb300 0.1 (sm_103a)"; }

mgs_status mgs_ctx_create(int32_t device, mgs_ctx *out) {
    if (!out) return fail(MGS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(MGS_ERR_INVALID_ARG, "no CUDA device %d", device);
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor < 100)
        return fail(MGS_ERR_INVALID_ARG, "device %d is sm_%d%d; this library is built for sm_103a",
                    device, prop.major, prop.minor);
    mgs_ctx c = new mgs_ctx_s;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    *out = c;
    return MGS_OK;
}

mgs_status mgs_ctx_destroy(mgs_ctx ctx) {
    delete ctx;
    return MGS_OK;
}

mgs_status mgs_ctx_info(mgs_ctx ctx, int32_t *sm_count, int64_t *free_bytes, int64_t *total_bytes) {
    if (!ctx) return fail(MGS_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    if (sm_count) *sm_count = ctx->sm_count;
    if (free_bytes) *free_bytes = (int64_t)fr;
    if (total_bytes) *total_bytes = (int64_t)tot;
    return MGS_OK;
}

mgs_status mgs_load_scene(mgs_ctx ctx, const mgs_scene_desc *d, mgs_stream stream_, mgs_scene *out) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!ctx || !d || !out) return fail(MGS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (d->n < 0 || d->n > (int64_t)1 << 31)
        return fail(MGS_ERR_INVALID_ARG, "n = %lld outside 0..2^31", (long long)d->n);
    if (d->precision != MGS_PREC_FP32 && d->precision != MGS_PREC_FP16)
        return fail(MGS_ERR_INVALID_ARG, "unknown precision %d", d->precision);
    if (d->order < MGS_ORDER_AUTO || d->order > MGS_ORDER_AS_GIVEN)
        return fail(MGS_ERR_INVALID_ARG, "unknown storage order %d", d->order);
    if (d->n > 0 && !d->attrs) return fail(MGS_ERR_INVALID_ARG, "attrs is NULL");
    const size_t elem = d->precision == MGS_PREC_FP16 ? 2 : 4;
    if (d->attrs_on_device && (reinterpret_cast<uintptr_t>(d->attrs) & 15))
        return fail(MGS_ERR_INVALID_ARG, "device attrs must be 16-byte aligned");
    const bool any_mlp = d->mlp_w1 || d->mlp_b1 || d->mlp_w2 || d->mlp_b2 || d->mlp_w3 || d->mlp_b3;
    const bool all_mlp = d->mlp_w1 && d->mlp_b1 && d->mlp_w2 && d->mlp_b2 && d->mlp_w3 && d->mlp_b3;
    if (any_mlp && !all_mlp) return fail(MGS_ERR_INVALID_ARG, "MLP weights are partially given");
    const int h1 = d->mlp_hidden[0], h2 = d->mlp_hidden[1], h3 = d->mlp_hidden[2];
    const bool wide = h1 != 0 || h2 != 0 || h3 != 0;
    if (wide) {
        for (int h : {h1, h2, h3})
            if (h < 16 || h > 256 || h % 16 != 0)
                return fail(MGS_ERR_INVALID_ARG, "MLP widths must be multiples of 16 in 16..256");
        if (!all_mlp || !d->mlp_w4 || !d->mlp_b4)
            return fail(MGS_ERR_INVALID_ARG, "the paper-width MLP needs w1..w4 and b1..b4");
        if (wide_mlp_smem(h1, h2, h3) > 227 * 1024)
            return fail(MGS_ERR_INVALID_ARG, "MLP widths %d/%d/%d exceed shared memory", h1, h2, h3);
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(MGS_ERR_CUDA, "cannot select device %d", ctx->device);

    mgs_scene s = new mgs_scene_s;
    s->ctx = ctx;
    s->n = d->n;
    s->precision = d->precision;
    const size_t bytes = (size_t)d->n * kRec * elem;
    const bool spatial = d->n > 1 && (d->order == MGS_ORDER_SPATIAL ||
                                      (d->order == MGS_ORDER_AUTO && d->n > (int64_t(1) << 21)));
    cudaError_t e = cudaMalloc(&s->attrs, bytes ? bytes : 16);
    if (e == cudaSuccess && spatial) e = cudaMalloc(&s->perm, (size_t)d->n * 4);
    if (e == cudaSuccess && spatial) e = cudaMalloc(&s->iperm, (size_t)d->n * 4);
    if (e != cudaSuccess) {
        dev_free(s->perm);
        dev_free(s->iperm);
        if (s->attrs) cudaFree(s->attrs);
        delete s;
        return cuda_fail(e, "scene allocation");
    }
    const cudaMemcpyKind kind = d->attrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (bytes && spatial) {
        // upload, then store in spatial (Morton) order
        void *tmp = nullptr;
        e = cudaMalloc(&tmp, bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, d->attrs, bytes, kind, stream);
        if (e == cudaSuccess) e = spatial_order(tmp, d->n, d->precision, s->attrs, s->perm, s->iperm, stream);
        if (tmp) cudaFree(tmp);
    } else if (bytes) {
        e = cudaMemcpyAsync(s->attrs, d->attrs, bytes, kind, stream);
    }
    s->bytes = (int64_t)bytes + (spatial ? (int64_t)d->n * 8 : 0);
    if (e == cudaSuccess && all_mlp && wide) {
        // pack: w1 [h1][32] (cols 22.. zero), w2 [h2][h1], w3 [h3][h2],
        // w4 [8][h3] (rows 5.. zero), then FP32 b1 [h1], b2 [h2], b3 [h3], b4 [8]
        const size_t n_w1 = (size_t)h1 * kMlpK1, n_w2 = (size_t)h2 * h1, n_w3 = (size_t)h3 * h2,
                     n_w4 = (size_t)kMlpN3 * h3;
        const size_t off_w2 = n_w1 * 2, off_w3 = off_w2 + n_w2 * 2, off_w4 = off_w3 + n_w3 * 2,
                     off_b1 = (off_w4 + n_w4 * 2 + 15) / 16 * 16, off_b2 = off_b1 + h1 * 4,
                     off_b3 = off_b2 + h2 * 4, off_b4 = off_b3 + h3 * 4, total = off_b4 + 8 * 4;
        std::vector<unsigned char> blob(total, 0);
        uint16_t *w1 = reinterpret_cast<uint16_t *>(blob.data());
        for (int r = 0; r < h1; ++r)
            for (int c = 0; c < kMlpIn; ++c) w1[r * kMlpK1 + c] = d->mlp_w1[r * kMlpIn + c];
        memcpy(blob.data() + off_w2, d->mlp_w2, n_w2 * 2);
        memcpy(blob.data() + off_w3, d->mlp_w3, n_w3 * 2);
        memcpy(blob.data() + off_w4, d->mlp_w4, (size_t)kMlpOut * h3 * 2);
        memcpy(blob.data() + off_b1, d->mlp_b1, h1 * 4);
        memcpy(blob.data() + off_b2, d->mlp_b2, h2 * 4);
        memcpy(blob.data() + off_b3, d->mlp_b3, h3 * 4);
        memcpy(blob.data() + off_b4, d->mlp_b4, kMlpOut * 4);
        e = cudaMalloc(&s->mlp_blob, total);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->mlp_blob, blob.data(), total, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        s->mlp.w1 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob);
        s->mlp.w2 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob + off_w2);
        s->mlp.w3 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob + off_w3);
        s->mlp.w4 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob + off_w4);
        s->mlp.b1 = reinterpret_cast<const float *>(s->mlp_blob + off_b1);
        s->mlp.b2 = reinterpret_cast<const float *>(s->mlp_blob + off_b2);
        s->mlp.b3 = reinterpret_cast<const float *>(s->mlp_blob + off_b3);
        s->mlp.b4 = reinterpret_cast<const float *>(s->mlp_blob + off_b4);
        s->mlp.h1 = h1;
        s->mlp.h2 = h2;
        s->mlp.h3 = h3;
        s->has_mlp = true;
        s->bytes += (int64_t)total;
    } else if (e == cudaSuccess && all_mlp) {
        // pack: w1 [64][32] (cols 22.. zero), w2 [64][64], w3 [8][64] (rows 5.. zero)
        const size_t n_w1 = kMlpHidden * kMlpK1, n_w2 = kMlpHidden * kMlpHidden,
                     n_w3 = kMlpN3 * kMlpHidden;
        const size_t off_w2 = n_w1 * 2, off_w3 = off_w2 + n_w2 * 2, off_b1 = off_w3 + n_w3 * 2,
                     off_b2 = off_b1 + 64 * 4, off_b3 = off_b2 + 64 * 4, total = off_b3 + 8 * 4;
        std::vector<unsigned char> blob(total, 0);
        uint16_t *w1 = reinterpret_cast<uint16_t *>(blob.data());
        uint16_t *w2 = reinterpret_cast<uint16_t *>(blob.data() + off_w2);
        uint16_t *w3 = reinterpret_cast<uint16_t *>(blob.data() + off_w3);
        float *b1 = reinterpret_cast<float *>(blob.data() + off_b1);
        float *b2 = reinterpret_cast<float *>(blob.data() + off_b2);
        float *b3 = reinterpret_cast<float *>(blob.data() + off_b3);
        for (int r = 0; r < kMlpHidden; ++r)
            for (int c = 0; c < kMlpIn; ++c) w1[r * kMlpK1 + c] = d->mlp_w1[r * kMlpIn + c];
        memcpy(w2, d->mlp_w2, n_w2 * 2);
        memcpy(w3, d->mlp_w3, (size_t)kMlpOut * kMlpHidden * 2);
        memcpy(b1, d->mlp_b1, 64 * 4);
        memcpy(b2, d->mlp_b2, 64 * 4);
        memcpy(b3, d->mlp_b3, kMlpOut * 4);
        e = cudaMalloc(&s->mlp_blob, total);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->mlp_blob, blob.data(), total, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        s->mlp.w1 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob);
        s->mlp.w2 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob + off_w2);
        s->mlp.w3 = reinterpret_cast<const __nv_bfloat16 *>(s->mlp_blob + off_w3);
        s->mlp.b1 = reinterpret_cast<const float *>(s->mlp_blob + off_b1);
        s->mlp.b2 = reinterpret_cast<const float *>(s->mlp_blob + off_b2);
        s->mlp.b3 = reinterpret_cast<const float *>(s->mlp_blob + off_b3);
        s->has_mlp = true;
        s->bytes += (int64_t)total;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        dev_free(s->mlp_blob);
        dev_free(s->perm);
        dev_free(s->iperm);
        cudaFree(s->attrs);
        delete s;
        return cuda_fail(e, "scene upload");
    }
    *out = s;
    return MGS_OK;
}

mgs_status mgs_unload_scene(mgs_scene s) {
    if (!s) return MGS_OK;
    DeviceGuard g(s->ctx->device);
    cudaFree(s->attrs);
    dev_free(s->mlp_blob);
    dev_free(s->perm);
    dev_free(s->iperm);
    delete s;
    return MGS_OK;
}

int64_t mgs_scene_bytes(mgs_scene s) { return s ? s->bytes : 0; }

mgs_status mgs_workspace_create(mgs_ctx ctx, mgs_workspace *out) {
    if (!ctx || !out) return fail(MGS_ERR_INVALID_ARG, "NULL argument");
    mgs_workspace w = new mgs_workspace_s;
    w->ctx = ctx;
    *out = w;
    return MGS_OK;
}

mgs_status mgs_workspace_destroy(mgs_workspace w) {
    if (!w) return MGS_OK;
    DeviceGuard g(w->ctx->device);
    dev_free(w->rec);
    dev_free(w->rect);
    dev_free(w->wt16);
    dev_free(w->tile_count);
    dev_free(w->tile_offsets);
    dev_free(w->tile_order);
    dev_free(w->gids);
    dev_free(w->bases);
    dev_free(w->img);
    dev_free(w->bwd_g);
    dev_free(w->bwd_partials);
    dev_free(w->ss.nkeys);
    dev_free(w->ss.nkeys_tmp);
    dev_free(w->ss.nvals);
    dev_free(w->ss.nvals_tmp);
    dev_free(w->ss.rank);
    dev_free(w->ss.keys);
    dev_free(w->ss.keys_tmp);
    dev_free(w->ss.vals);
    dev_free(w->ss.vals_tmp);
    if (w->ss.temp) cudaFree(w->ss.temp);
    dev_free(w->status);
    for (auto &q : w->pending)
        for (auto x : q) cudaEventDestroy(x);
    for (auto x : w->event_pool) cudaEventDestroy(x);
    delete w;
    return MGS_OK;
}

mgs_status mgs_workspace_reserve(mgs_workspace w, int64_t n, int32_t width, int32_t height,
                                 int64_t pairs) {
    if (!w) return fail(MGS_ERR_INVALID_ARG, "workspace is NULL");
    if (n < 0 || pairs < 0 || width < 1 || height < 1 || width > 16384 || height > 16384)
        return fail(MGS_ERR_INVALID_ARG, "bad reserve sizes");
    DeviceGuard g(w->ctx->device);
    const int64_t T = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
    return ws_ensure(w, n, T, (uint64_t)pairs);
}

int64_t mgs_workspace_bytes(mgs_workspace w) { return w ? ws_bytes(w) : 0; }

mgs_status mgs_workspace_sync(mgs_workspace w, mgs_stream stream_, int64_t *pairs_out) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!w) return fail(MGS_ERR_INVALID_ARG, "workspace is NULL");
    DeviceGuard g(w->ctx->device);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (pairs_out) *pairs_out = 0;
    if (!w->status) return MGS_OK;
    DevStatus h;
    if ((e = cudaMemcpy(&h, w->status, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    if ((e = cudaMemset(w->status, 0, offsetof(DevStatus, last_pairs))) != cudaSuccess)
        return cuda_fail(e, "status reset");
    if (pairs_out) *pairs_out = (int64_t)h.max_pairs;
    if (h.overflow & kStatusMmaTimeout)
        return fail(MGS_ERR_TIMEOUT, "a tensor-core MMA wait in preprocessing timed out");
    if (h.overflow & kStatusOverflow) {
        uint64_t need = h.max_pairs + h.max_pairs / 4 + 1024;
        if (w->grow_hint < need) w->grow_hint = need;
        return fail(MGS_ERR_OVERFLOW, "tile lists needed %llu pairs, capacity was %llu",
                    (unsigned long long)h.max_pairs, (unsigned long long)w->pair_cap);
    }
    return MGS_OK;
}

mgs_status mgs_workspace_set_timing(mgs_workspace w, int32_t enable) {
    if (!w) return fail(MGS_ERR_INVALID_ARG, "workspace is NULL");
    w->timing = enable != 0;
    return MGS_OK;
}

mgs_status mgs_workspace_stage_times(mgs_workspace w, mgs_stream stream_, double ms[6],
                                     int64_t *frames) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!w || !ms || !frames) return fail(MGS_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(w->ctx->device);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    for (int k = 0; k < kStageEvents - 1; ++k) ms[k] = 0.0;
    *frames = (int64_t)w->pending.size();
    for (auto &q : w->pending) {
        for (int k = 0; k < kStageEvents - 1; ++k) {
            float t = 0.f;
            if ((e = cudaEventElapsedTime(&t, q[k], q[k + 1])) != cudaSuccess)
                return cuda_fail(e, "event elapsed time");
            ms[k] += t;
        }
        for (auto x : q) w->event_pool.push_back(x);
    }
    w->pending.clear();
    return MGS_OK;
}

mgs_status mgs_render(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                      const mgs_render_opts *opts, float *out_rgb, float *out_aux,
                      int32_t *out_count, mgs_stream stream) {
    return render_impl(w, s, cam, opts, out_rgb, out_aux, out_count,
                       reinterpret_cast<cudaStream_t>(stream));
}

mgs_status mgs_render_depth(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                            const mgs_render_opts *opts, float *out_rgb, float *out_depth,
                            mgs_stream stream) {
    if (!out_depth) return fail(MGS_ERR_INVALID_ARG, "out_depth is NULL");
    return render_impl(w, s, cam, opts, out_rgb, nullptr, nullptr,
                       reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, out_depth);
}

mgs_status mgs_render_backward(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                               const mgs_render_opts *opts, const float *dL_drgb,
                               const float *aux, float *d_attrs, float *d_mlp,
                               mgs_stream stream) {
    if (!dL_drgb || !aux || !d_attrs)
        return fail(MGS_ERR_INVALID_ARG, "dL_drgb, aux and d_attrs are required");
    if (opts && opts->use_mlp == 0 && d_mlp == nullptr) {
        // fine: no MLP gradients requested
    }
    BackwardIO io{dL_drgb, aux, d_attrs, d_mlp};
    return render_impl(w, s, cam, opts, nullptr, nullptr, nullptr,
                       reinterpret_cast<cudaStream_t>(stream), &io);
}

mgs_status mgs_render_checked(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                              const mgs_render_opts *opts, float *out_rgb, float *out_aux,
                              int32_t *out_count, mgs_stream stream) {
    for (int attempt = 0; attempt < 2; ++attempt) {
        mgs_status st = mgs_render(w, s, cam, opts, out_rgb, out_aux, out_count, stream);
        if (st != MGS_OK) return st;
        st = mgs_workspace_sync(w, stream, nullptr);
        if (st != MGS_ERR_OVERFLOW) return st;
    }
    return MGS_ERR_OVERFLOW;
}

mgs_status mgs_render_to_host(mgs_workspace w, mgs_scene s, const mgs_camera *cam,
                              const mgs_render_opts *opts, float *host_rgb, mgs_stream stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!w) return fail(MGS_ERR_INVALID_ARG, "workspace is NULL");
    if (!host_rgb) return fail(MGS_ERR_INVALID_ARG, "host_rgb is NULL");
    mgs_status st = check_camera(cam);
    if (st != MGS_OK) return st;
    DeviceGuard g(w->ctx->device);
    const int64_t px = (int64_t)cam->width * cam->height;
    if (px > w->img_cap) {
        dev_free(w->img);
        w->img_cap = 0;
        cudaError_t e = dev_alloc(&w->img, (size_t)px * 3);
        if (e != cudaSuccess) return cuda_fail(e, "workspace image");
        w->img_cap = px;
    }
    st = render_impl(w, s, cam, opts, w->img, nullptr, nullptr, stream);
    if (st != MGS_OK) return st;
    cudaError_t e = cudaMemcpyAsync(host_rgb, w->img, (size_t)px * 12, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "image copy");
    return MGS_OK;
}

mgs_status mgs_frame_stats(mgs_workspace w, mgs_stream stream_, int64_t *visible,
                           int64_t *pairs, int64_t *fp32_sum_tiles) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!w || !visible || !pairs || !fp32_sum_tiles) return fail(MGS_ERR_INVALID_ARG, "NULL argument");
    *visible = *pairs = *fp32_sum_tiles = 0;
    if (!w->status || w->last_tiles == 0) return fail(MGS_ERR_INVALID_ARG, "no render yet");
    DeviceGuard g(w->ctx->device);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    DevStatus h;
    if ((e = cudaMemcpy(&h, w->status, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    *visible = (int64_t)h.last_visible;
    *pairs = (int64_t)h.last_pairs;
    *fp32_sum_tiles = (int64_t)h.last_wide_tiles;
    return MGS_OK;
}

mgs_status mgs_tile_lists(mgs_workspace w, mgs_stream stream_, int64_t *n_tiles,
                          int64_t *n_pairs, uint32_t *offsets_out, uint32_t *gids_out) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!w || !n_tiles || !n_pairs) return fail(MGS_ERR_INVALID_ARG, "NULL argument");
    *n_tiles = *n_pairs = 0;
    if (!w->status || w->last_tiles == 0) return fail(MGS_ERR_INVALID_ARG, "no render yet");
    DeviceGuard g(w->ctx->device);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    DevStatus h;
    if ((e = cudaMemcpy(&h, w->status, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "status read");
    *n_tiles = w->last_tiles;
    *n_pairs = (int64_t)h.last_pairs;
    if (h.last_pairs > w->pair_cap)
        return fail(MGS_ERR_OVERFLOW, "the last render overflowed its tile lists");
    if (offsets_out && gids_out) {
        e = cudaMemcpy(offsets_out, w->tile_offsets, (size_t)(w->last_tiles + 1) * 4,
                       cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess && h.last_pairs) {
            // list entries index the scene's stored (spatial) order: report caller indices
            e = w->last_perm ? map_ids(w->gids, w->last_perm, (int64_t)h.last_pairs, gids_out, stream)
                             : cudaMemcpy(gids_out, w->gids, (size_t)h.last_pairs * 4,
                                          cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "tile list copy");
    }
    return MGS_OK;
}

}  // extern "C"
