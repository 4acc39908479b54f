/*
 * mobilegs.h -- C-ABI of the GB300 (sm_103a) sort-free Gaussian renderer.
 *
 * The renderer computes the depth-aware, order-independent image of Mobile-GS
 * (arxiv 2603.11531):
 *
 *   C(p) = (1 - T) * sum_i c_i a_i w_i / sum_i a_i w_i + T * c_bg      (Sec. 3.1, Eq. 2)
 *   T    = prod_i (1 - a_i),   a_i = o_i exp(-1/2 dx^T Sigma_i^-1 dx)  (Sec. 3.1, Eq. 2)
 *   w_i  = phi_i^2 + phi_i / d_i^2 + exp(s_max / d_i)                 (Sec. 3.1, Eq. 3)
 *   phi_i, o_i = ReLU(MLP_phi F), sigmoid(MLP_o F),
 *   F = MLP_f(P_i, s_i, r_i, Y_i)                                      (Sec. 3.1, Eq. 4)
 *
 * with c_i the first-order spherical-harmonics colour (Sec. 3.2) and the
 * Gaussians (mu, Sigma = R S S^T R^T, o, Y) projected as in App. B.  The sums
 * commute (Sec. 2, discussion of Eq. 1), so no depth sort is done: Gaussians
 * are binned into 16x16-pixel tiles by tile only, and every pixel
 * accumulates its tile's list in whatever order it is stored.
 *
 * Conventions for every entry point:
 *   - Every function returns an mgs_status; nothing throws across the ABI.
 *     On failure, mgs_last_error() returns a message for the calling thread.
 *   - Device pointers are CUDA global-memory pointers on the context's
 *     device; host pointers are ordinary (pageable or pinned) memory.
 *   - Output buffers are owned by the caller; the library never frees them.
 *     Scenes and workspaces own their device memory until destroyed.
 *   - Rendering calls are asynchronous on the given stream (NULL = the legacy
 *     default stream).  Arguments are checked on the host before any launch.
 *     Errors that only the device can see (tile-list capacity overflow, a
 *     tensor-core wait that ran out) are recorded in the workspace and
 *     reported by mgs_workspace_sync().
 *   - A workspace holds the per-frame scratch (projected Gaussians, tile
 *     lists).  Renders that share a workspace must be ordered on one stream;
 *     concurrent renders need one workspace each.
 */
#ifndef MOBILEGS_H
#define MOBILEGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (same type, declared here so that this header needs no CUDA
 * headers). */
typedef struct CUstream_st *mgs_stream;

typedef enum {
    MGS_OK = 0,
    MGS_ERR_INVALID_ARG = 1,  /* bad pointer, size, camera or option */
    MGS_ERR_OOM = 2,          /* device allocation failed */
    MGS_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
    MGS_ERR_OVERFLOW = 4,     /* a render needed more tile-list capacity than
                                 its workspace had; its image is invalid */
    MGS_ERR_TIMEOUT = 5,      /* a bounded wait gave up */
    MGS_ERR_BUSY = 6,         /* resource in use (e.g. admission refused) */
    MGS_ERR_NOT_READY = 7     /* work still in flight */
} mgs_status;

enum { MGS_PREC_FP32 = 0, MGS_PREC_FP16 = 1 };

/* Render flags (mgs_render_opts.flags). */
enum {
    MGS_FLAG_NO_CULL = 1u, /* debug: skip the conservative per-warp culling of
                              tile lists (the image must not change) */
    MGS_FLAG_MLP_MMA_SYNC = 4u, /* run the MLP on warp-level mma.sync instead
                              of tcgen05 (comparison and testing) */
    MGS_FLAG_RASTER_FMA = 8u, /* FP16 scenes: accumulate A and B on the FP32
                              FMA pipe instead of the tensor cores (exact
                              FP32 sums, slower; comparison and testing) */
    MGS_FLAG_SORTED = 2u   /* comparator, not the paper's method: depth-sort
                              every tile list (radix sort) and alpha-blend
                              front to back, C = sum c_i a_i T_i + T c_bg
                              (App. B, Eq. 11, 3DGS early termination at
                              T < 1e-4); out_aux must be NULL */
};

typedef struct mgs_ctx_s *mgs_ctx;
typedef struct mgs_scene_s *mgs_scene;
typedef struct mgs_workspace_s *mgs_workspace;

/* Gaussian record: 24 elements of the stored precision per Gaussian (App. B
 * parameters; activated values):
 *   [0..2]  mean mu (world)          [3..5]  scale s (> 0, per local axis)
 *   [6..9]  quaternion (w, x, y, z), any norm > 0 (normalised by the renderer)
 *   [10]    opacity o in [0, 1]      [11..22] SH coefficients, coefficient-
 *                                          major: Y0 rgb, Y1 rgb, Y2 rgb, Y3 rgb
 *   [23]    ignored (padding)
 * Enhancement MLP (Eq. 4), optional: w1 [64][22], w2 [64][64], w3 [5][64]
 * as BF16 bit patterns, row-major [out][in]; biases b1 [64], b2 [64], b3 [5]
 * FP32.  Head rows: phi, o, d_r, d_g, d_b (the last three are an optional
 * colour residual).  MLP input: [P(3), s(3), normalised q(4), Y(12)].
 * Paper-width MLP_f (App. C: 256, 128, 64 neurons): set mlp_hidden to the
 * three widths (each a multiple of 16 in 16..256); then w1 [h1][22],
 * w2 [h2][h1], w3 [h3][h2] are the hidden layers, w4 [5][h3] the head, and
 * b1..b4 their biases.  It runs on tcgen05 only and has no backward pass.
 * mlp_hidden all zero: the 22 -> 64 -> 64 -> 5 MLP (w4, b4 unused). */
typedef struct {
    int64_t n;              /* number of Gaussians, >= 0 */
    int32_t precision;      /* MGS_PREC_FP32 or MGS_PREC_FP16 */
    int32_t attrs_on_device;/* 1: attrs is a device pointer; 0: host */
    const void *attrs;      /* n x 24 elements, 16-byte aligned if on device */
    const uint16_t *mlp_w1; /* host pointers; all NULL = scene has no MLP */
    const float *mlp_b1;
    const uint16_t *mlp_w2;
    const float *mlp_b2;
    const uint16_t *mlp_w3;
    const float *mlp_b3;
    const uint16_t *mlp_w4; /* head of the paper-width MLP, else NULL */
    const float *mlp_b4;
    int32_t mlp_hidden[3];  /* {0, 0, 0} or three hidden widths */
    int32_t order;          /* storage order, MGS_ORDER_* (0: automatic) */
} mgs_scene_desc;

/* Storage order of a loaded scene.  Spatial order (a Morton curve of the
 * means) keeps the tile-list writes of binning local, which pays once the
 * lists outgrow the L2 cache; for smaller scenes the given (random) order
 * spreads binning's shared-memory atomics better.  Automatic: spatial above
 * 2^21 Gaussians. */
enum { MGS_ORDER_AUTO = 0, MGS_ORDER_SPATIAL = 1, MGS_ORDER_AS_GIVEN = 2 };

/* Pinhole camera, world->camera (R row-major, t), OpenCV axes (x right,
 * y down, z forward).  Pixel (x, y) has its centre at (x + 0.5, y + 0.5). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;   /* 1 .. 16384 */
    float znear;             /* > 0: Gaussians with view z <= znear are culled */
} mgs_camera;

typedef struct {
    int32_t use_mlp;          /* 0: phi = 1, o = stored opacity; 1: Eq. 4 */
    int32_t mlp_rgb_residual; /* 1: add the MLP's colour head before clamping */
    float bg[3];              /* c_bg */
    uint32_t flags;           /* MGS_FLAG_* */
} mgs_render_opts;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`. */
mgs_status mgs_ctx_create(int32_t device, mgs_ctx *out);
mgs_status mgs_ctx_destroy(mgs_ctx ctx);

/* Static facts of the context's device: SM count, free and total memory. */
mgs_status mgs_ctx_info(mgs_ctx ctx, int32_t *sm_count, int64_t *free_bytes,
                        int64_t *total_bytes);

/* ---- scenes (App. B parameters, resident in device memory) --------------- */

/* Copy a scene into library-owned device memory (stream-ordered on
 * `stream`; the copy has completed when the call returns, so host buffers
 * may be reused at once).  MLP weights are repacked for the tensor cores.
 * The library may store the Gaussians in its own order (desc->order);
 * images do not depend on it, and every per-Gaussian output (tile lists,
 * gradients) uses the caller's indices. */
mgs_status mgs_load_scene(mgs_ctx ctx, const mgs_scene_desc *desc,
                          mgs_stream stream, mgs_scene *out);
mgs_status mgs_unload_scene(mgs_scene scene);
/* Device bytes held by the scene. */
int64_t mgs_scene_bytes(mgs_scene scene);

/* ---- workspaces (per-frame scratch) -------------------------------------- */

mgs_status mgs_workspace_create(mgs_ctx ctx, mgs_workspace *out);
mgs_status mgs_workspace_destroy(mgs_workspace ws);
/* Pre-size the scratch for n Gaussians, a width x height image and `pairs`
 * (tile, Gaussian) intersections, so that later renders allocate nothing. */
mgs_status mgs_workspace_reserve(mgs_workspace ws, int64_t n, int32_t width,
                                 int32_t height, int64_t pairs);
/* Device bytes held by the workspace. */
int64_t mgs_workspace_bytes(mgs_workspace ws);
/* Wait for `stream`, then report renders since the previous sync:
 * MGS_ERR_OVERFLOW if any ran out of tile-list capacity (the workspace is then
 * grown so that a repeat succeeds); MGS_ERR_TIMEOUT if a tensor-core MMA wait
 * in the MLP gave up (that image is invalid; checked first).  *pairs_out
 * (nullable) = the largest number of (tile, Gaussian) pairs any of them
 * needed. */
mgs_status mgs_workspace_sync(mgs_workspace ws, mgs_stream stream,
                              int64_t *pairs_out);

/* Per-stage device timing (the runtime breakdown the paper reports in
 * Fig. 2 and Fig. 6).  While enabled, every render on the workspace records
 * CUDA events on its stream around (0) preprocessing incl. the MLP, the four
 * parts of binning -- (1) the work plan (count reset, pair counts per group,
 * plan scan), (2) the tile count, (3) the tile scan and rasterisation order,
 * (4) the scatter of the lists -- and (5) rasterisation (the sorted
 * comparator's sort and blend; the backward pass's adjoint). */
mgs_status mgs_workspace_set_timing(mgs_workspace ws, int32_t enable);
/* Wait for `stream`; ms[0..5] = summed stage times in milliseconds of the
 * renders timed since the previous call, *frames = their number.  Resets. */
mgs_status mgs_workspace_stage_times(mgs_workspace ws, mgs_stream stream,
                                     double ms[6], int64_t *frames);

/* ---- rendering (Sec. 3.1, Eq. 2-4) --------------------------------------- */

/* Render one view.  out_rgb: device, height x width x 3 FP32 (row-major, RGB
 * interleaved).  out_aux (nullable): device, 5 x height x width FP32 planes
 * (A_r, A_g, A_b, B, T) with A = sum c a w, B = sum a w, T = prod (1 - a),
 * the quantities the backward pass needs.  out_count (nullable): device,
 * height x width int32, number of Gaussians included at each pixel.
 * Asynchronous; a capacity overflow is reported by mgs_workspace_sync(). */
mgs_status mgs_render(mgs_workspace ws, mgs_scene scene, const mgs_camera *cam,
                      const mgs_render_opts *opts, float *out_rgb,
                      float *out_aux, int32_t *out_count, mgs_stream stream);

/* mgs_render, then mgs_workspace_sync, repeated once after growing the
 * workspace if the first attempt overflowed.  Synchronous. */
mgs_status mgs_render_checked(mgs_workspace ws, mgs_scene scene,
                              const mgs_camera *cam,
                              const mgs_render_opts *opts, float *out_rgb,
                              float *out_aux, int32_t *out_count,
                              mgs_stream stream);

/* Depth image for the depth distillation of Sec. 3.2 (Eq. 5): renders the
 * colour image into out_rgb (as mgs_render) and the depth-aware weighted mean
 * view depth D = sum d_i a_i w_i / sum a_i w_i (Eq. 2's weights; 0 where no
 * Gaussian is included) into out_depth (device, height x width FP32).  The
 * colour image equals mgs_render's with the same options.  The numerator
 * sum d a w is FP32; the denominator sum a w is FP32 for FP32 attributes
 * (or MGS_FLAG_RASTER_FMA) and the tensor-core B of the colour image for
 * FP16 attributes.  MGS_FLAG_SORTED is not accepted.
 * Errors: MGS_ERR_INVALID_ARG for a NULL out_depth, otherwise as mgs_render. */
mgs_status mgs_render_depth(mgs_workspace ws, mgs_scene scene,
                            const mgs_camera *cam, const mgs_render_opts *opts,
                            float *out_rgb, float *out_depth, mgs_stream stream);

/* Load-time SH decoder of Sec. 3.2, Eq. 6 (one of MLP_d, MLP_v): 6 inputs
 * (h_d, h_v) -> 64 ReLU units -> n_out outputs (3 for MLP_d, 9 for MLP_v),
 * every parameter an IEEE binary16 bit pattern (App. C: 16-bit MLPs),
 * row-major [out][in].  Host pointers, read during the call. */
typedef struct {
    const uint16_t *w1;   /* [64][6] */
    const uint16_t *b1;   /* [64] */
    const uint16_t *w2;   /* [n_out][64] */
    const uint16_t *b2;   /* [n_out] */
} mgs_sh_mlp;

/* Decodes the SH coefficients of n Gaussians once, before loading (Eq. 6):
 * f_d = MLP_d(h_d, h_v) is written to attribute columns 11..13 (Y0 rgb) and
 * f_v = MLP_v(h_d, h_v) to columns 14..22 (Y1 rgb, Y2 rgb, Y3 rgb) of the
 * device array attrs (n x 24 elements of `precision`, other columns left
 * untouched); h is a device array of n x 6 elements of `precision`.  FP32
 * accumulation; FP16 attributes receive the result rounded to nearest.
 * Asynchronous on `stream`; MGS_ERR_INVALID_ARG for NULL or bad arguments. */
mgs_status mgs_decode_sh(mgs_ctx ctx, int64_t n, int32_t precision,
                         const void *h, const mgs_sh_mlp *mlp_d,
                         const mgs_sh_mlp *mlp_v, void *attrs,
                         mgs_stream stream);

/* End-to-end render into HOST memory: renders into a workspace-owned device
 * image and copies it to host_rgb (height x width x 3 FP32; pinned memory
 * gives an asynchronous copy).  Asynchronous on `stream` like mgs_render. */
mgs_status mgs_render_to_host(mgs_workspace ws, mgs_scene scene,
                              const mgs_camera *cam,
                              const mgs_render_opts *opts, float *host_rgb,
                              mgs_stream stream);

/* Tile lists of the workspace's most recent render, for tests.  Waits for
 * `stream`, then reports n_tiles and n_pairs (= offsets[n_tiles]); if both
 * output buffers are non-NULL it also copies offsets [n_tiles + 1] and
 * gids [n_pairs] into them (caller-owned device memory).  Gaussian indices
 * are the caller's (as in the scene description; the scene must still be
 * loaded), in unspecified order within a tile.  MGS_ERR_OVERFLOW if that
 * render overflowed (its lists are incomplete). */
mgs_status mgs_tile_lists(mgs_workspace ws, mgs_stream stream, int64_t *n_tiles,
                          int64_t *n_pairs, uint32_t *offsets_out,
                          uint32_t *gids_out);

/* Facts of the workspace's most recent render, for measurement: Gaussians
 * that passed culling (visible), listed (tile, Gaussian) pairs, and tiles
 * whose A, B sums ran in FP32 because they list a Gaussian whose Eq. 3 weight
 * the FP16 tensor-core sums cannot hold next to the others.  Waits for
 * `stream`.  MGS_ERR_INVALID_ARG before the first render. */
mgs_status mgs_frame_stats(mgs_workspace ws, mgs_stream stream, int64_t *visible,
                           int64_t *pairs, int64_t *fp32_sum_tiles);

/* ---- differentiation (adjoint of Sec. 3.1 Eq. 2-4, Sec. 3.2, App. B) ------- */

/* Gradients of a loss L with respect to every stored Gaussian attribute and
 * the MLP parameters, given dL/dC of a render of the same view.
 *   dL_drgb: device, height x width x 3 FP32 (dL/dC).
 *   aux:     device, 5 x height x width FP32, the out_aux of mgs_render for
 *            this scene, camera and options (A_rgb, B, T).
 *   d_attrs: device, n x 24 FP32, overwritten with dL/d(record element) (the
 *            widened FP16 values for FP16 scenes; padding 0; the opacity
 *            column is 0 in MLP mode, where Eq. 4 replaces the stored opacity).
 *   d_mlp:   device, 5957 FP32 or NULL, overwritten with dL/dW1 [64][22],
 *            dL/db1 [64], dL/dW2 [64][64], dL/db2 [64], dL/dW3 [5][64],
 *            dL/db3 [5] (zeros without the MLP).  The BF16 rounding of the
 *            MLP's tensor-core inputs is passed straight through.
 * The inclusion test and tile rectangles are piecewise constant; their
 * derivative is taken as zero.  Asynchronous on `stream`; reuses the
 * workspace (it rebuilds the frame's records and tile lists). */
mgs_status mgs_render_backward(mgs_workspace ws, mgs_scene scene,
                               const mgs_camera *cam,
                               const mgs_render_opts *opts,
                               const float *dL_drgb, const float *aux,
                               float *d_attrs, float *d_mlp, mgs_stream stream);

/* ---- serving: continuous batching of render requests ------------------------ */

typedef struct mgs_server_s *mgs_server;

typedef struct {
    int32_t slots;             /* views in flight at once (1..64); each slot owns
                                  a workspace and a stream */
    int32_t max_batch;         /* views rasterised by one persistent launch (1..64) */
    int64_t hbm_budget_bytes;  /* device bytes the slots' workspaces may hold */
} mgs_server_config;

/* Start a server on the context's device.  A worker thread owned by the
 * server admits queued requests, in arrival order, into free slots while their
 * estimated scratch fits the budget.  Every slot works on its own stream, so
 * the requests in flight overlap on the device.  A view of more than 2,048
 * tiles runs alone: preprocessing, MLP, binning and rasterisation as one CUDA
 * graph.  Consecutive smaller views (up to max_batch) form a group: their
 * preprocessing and binning run as graphs on their slots' streams, and one
 * launch of the persistent batched rasteriser draws all their tiles.  Graphs
 * are instantiated once per (slot, scene, resolution, options) and relaunched
 * with the new camera and output set in the kernel nodes that read them.
 * Completion is recorded per group.  Not in the paper: the serving pattern of
 * the workload. */
mgs_status mgs_server_create(mgs_ctx ctx, const mgs_server_config *cfg, mgs_server *out);
/* Finish every queued and running request, then release the server. */
mgs_status mgs_server_destroy(mgs_server srv);
/* Queue one view of a resident scene; out_rgb (device, height x width x 3
 * FP32, caller-owned) must stay valid until the ticket completes.
 * Thread-safe. */
mgs_status mgs_server_submit(mgs_server srv, mgs_scene scene, const mgs_camera *cam,
                             const mgs_render_opts *opts, float *out_rgb, int64_t *ticket);
/* Wait at most timeout_ms for the ticket: MGS_ERR_TIMEOUT if it is not done,
 * else the request's own status (MGS_OK, or MGS_ERR_OOM if it can never fit
 * the budget). */
mgs_status mgs_server_wait(mgs_server srv, int64_t ticket, double timeout_ms);
/* A ticket's state (0 queued, 1 running, 2 done), status and steady-clock
 * timestamps in seconds (same clock as mgs_now): submitted, admitted, done. */
mgs_status mgs_server_ticket(mgs_server srv, int64_t ticket, int32_t *state, int32_t *result,
                             double *t_submit, double *t_admit, double *t_done);
/* Counters: completed, queued and running requests, workspace bytes held,
 * whether graphs are in use (1) or launches are direct (0). */
mgs_status mgs_server_stats(mgs_server srv, int64_t *completed, int64_t *queued,
                            int64_t *running, int64_t *workspace_bytes, int32_t *graphs);
/* The server's steady clock, in seconds. */
double mgs_now(void);

/* ---- allocation-free rendering -------------------------------------------- */

/* Renders one view without allocating any device memory, for callers that
 * cannot call cudaMalloc (code where the device allocator is forbidden or
 * unavailable, or a real-time loop that must not take its locks or fail on an
 * out-of-memory condition).  The paper has no counterpart: this is a
 * deployment variant of mgs_render.
 *   attrs:     device pointer, n x 24 records (same layout as mgs_scene_desc),
 *              16-byte aligned; precision MGS_PREC_FP32 or MGS_PREC_FP16.
 *   out_rgb:   device, height x width x 3 FP32, caller-owned.
 *   opts:      use_mlp must be 0 (plain mode: phi = 1, stored opacity);
 *              flags may hold only MGS_FLAG_NO_CULL and MGS_FLAG_RASTER_FMA
 *              (any other flag, e.g. MGS_FLAG_SORTED, is MGS_ERR_INVALID_ARG).
 * Scratch lives in one fixed __device__ array (30,557,440 bytes, about
 * 29 MiB) that every GPU loading this library holds until the process exits.  Limits: n <= 131072,
 * at most 8192 tiles of 16x16 pixels (1920x1080 fits), at most 4,194,304
 * (tile, Gaussian) pairs; larger n or images are rejected with
 * MGS_ERR_INVALID_ARG before any work, too many pairs with MGS_ERR_OVERFLOW
 * (the image is then invalid).  The call waits for `stream` before returning.
 * The first call on a device resolves the array's device address (set-up with
 * that device current); make it before any stream capture.  All calls share
 * the array, so calls whose GPU work overlaps race: order them on one stream
 * or serialise them. */
mgs_status mgs_render_static(const void *attrs, int64_t n, int32_t precision,
                             const mgs_camera *cam, const mgs_render_opts *opts,
                             float *out_rgb, mgs_stream stream);

/* ---- diagnostics --------------------------------------------------------- */

/* Measured issue rates of the two pipes that bound the rasteriser (Sec. 3.1,
 * Eq. 2: one exponential and about 16 FP32 operations per included
 * pixel-Gaussian pair), per SM per clock cycle on CUDA device `device`:
 * ex2.approx.ftz.f32 (MUFU) and FP32 FFMA.  Blocks of 256 threads run eight
 * independent dependency chains per thread and record their SM and first and
 * last cycle on its counter; per SM, operations over the span of its blocks,
 * averaged over the SMs.  Synchronous; allocates and frees two small device
 * buffers.  MGS_ERR_INVALID_ARG for NULL outputs or a bad device. */
mgs_status mgs_probe_rates(int32_t device, double *ex2_per_sm_clk, double *ffma_per_sm_clk);

/* Measured rate of scattered 4-byte stores, one 32-byte sector each, per SM
 * per clock cycle on CUDA device `device`: what bounds the list writes of
 * tile binning (Sec. 2: lists keyed by tile only, each (tile, Gaussian) entry
 * written to its tile's list, so consecutive entries of a warp land in
 * different sectors).  Blocks of 256 threads write 256 words each to
 * pseudo-random sector starts of a 64 MB device buffer (L2-resident, like the
 * lists); per SM, sectors over the span of its blocks, averaged over the SMs.
 * Synchronous; allocates and frees two device buffers.  MGS_ERR_INVALID_ARG
 * for a NULL output or a bad device. */
mgs_status mgs_probe_store(int32_t device, double *sectors_per_sm_clk);

const char *mgs_last_error(void);
const char *mgs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MOBILEGS_H */
