/*
 * FP64 CPU oracle for the Mobile-GS sort-free (depth-aware, order-independent)
 * Gaussian renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA renderer: only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code with the CUDA library and includes none of its
 * headers.
 *
 * What it computes (paper sections):
 *   - App. B: Gaussians (mu, Sigma = R S S^T R^T, o, Y), perspective
 *     projection; the projection/EWA details follow the 3DGS convention the
 *     paper inherits (App. B, Sec. 2).
 *   - Sec. 3.1, Eq. 2: C = (1 - T) * sum(c a w) / sum(a w) + T * c_bg,
 *     T = prod(1 - a), a = o * exp(-q / 2).
 *   - Sec. 3.1, Eq. 3: w = phi^2 + phi / d^2 + exp(s_max / d).
 *   - Sec. 3.1, Eq. 4: F = MLP_f(P, s, r, Y), phi = ReLU(MLP_phi F),
 *     o = sigmoid(MLP_o F), P = (mu - t_v) / |mu - t_v|.
 *   - Sec. 3.2: first-order (degree-1) SH colour.
 *
 * Values are FP64.  Which Gaussians exist in a frame, their 16x16-tile
 * rectangles and the per-pixel inclusion test are taken from a fixed
 * sequence of correctly rounded binary32 operations (the "FP32 contract",
 * mgs_oracle.c), so that tile lists can be compared bit-exactly as sets.
 */
#ifndef MGS_ORACLE_H
#define MGS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TILE 16
#define ORC_REC 24

/* Camera: world->camera rotation R (row-major) and translation t, pinhole
 * intrinsics; OpenCV axes (x right, y down, z forward).  Pixel (x, y) has its
 * centre at (x + 0.5, y + 0.5). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
} orc_camera;

/* Enhancement MLP (Eq. 4), head rows (phi, o, d_r, d_g, d_b).  Weights are
 * BF16 bit patterns, row-major [out][in]; biases FP32.
 *   h1 == 0: 22 -> 64 -> 64 -> 5, w3/b3 the head (w4/b4 unused);
 *   h1 != 0: 22 -> h1 -> h2 -> h3 -> 5, w4/b4 the head (App. C's MLP_f has
 *            h = 256, 128, 64). */
typedef struct {
    const uint16_t *w1; const float *b1;   /* [h1][22], [h1] */
    const uint16_t *w2; const float *b2;   /* [h2][h1], [h2] */
    const uint16_t *w3; const float *b3;   /* [h3][h2] (or the [5][64] head) */
    const uint16_t *w4; const float *b4;   /* [5][h3], [5] */
    int32_t h1, h2, h3;
    int32_t pad;
} orc_mlp;

/* Per-Gaussian result of the preprocessing stage. */
typedef struct {
    int32_t visible;    /* FP32 contract: survived the near-plane, determinant
                           and empty-rectangle culls */
    int32_t rect[4];    /* tile rectangle [x_lo, x_hi) x [y_lo, y_hi):
                           x_lo, y_lo, x_hi, y_hi */
    float   m32[2];     /* FP32 contract pixel mean */
    float   l32[3];     /* FP32 contract factors: q = (l11 dx + l21 dy)^2
                           + (l22 dy)^2 */
    float   tz32;       /* FP32 contract view depth (orders the sorted
                           comparator) */
    double  mean[2];    /* FP64 pixel mean */
    double  cov[3];     /* FP64 Sigma_2D (a, b, c), dilation included */
    double  conic[3];   /* FP64 inverse of Sigma_2D (A, B, C) */
    double  depth;      /* view-space z */
    double  rgb[3];     /* colour c_i */
    double  opacity;    /* o_i */
    double  phi;        /* phi_i */
    double  weight;     /* w_i (Eq. 3) */
    double  dir[3];     /* P_i */
} orc_gauss;

int64_t orc_gauss_size(void);

/* Rotation matrix (row-major) of the normalised quaternion q = (w, x, y, z). */
void orc_rotation(const double q[4], double R[9]);

/* Load-time SH decode of Sec. 3.2, Eq. 6: f_d = MLP_d(h_d, h_v) (3 values,
 * the degree-0 colour coefficients) and f_v = MLP_v(h_d, h_v) (9 values, the
 * degree-1 coefficients Y1 rgb, Y2 rgb, Y3 rgb).  Each MLP has one hidden
 * layer of 64 ReLU units (App. C) and 16-bit parameters: w1 [64][6],
 * b1 [64], w2 [n_out][64], b2 [n_out] as IEEE binary16 bit patterns. */
typedef struct {
    const uint16_t *w1, *b1, *w2, *b2;
    int32_t n_out;
    int32_t pad;
} orc_sh_mlp;

/* h: n x 6 (h_d, h_v); Y: n x 12 SH coefficients, coefficient-major
 * (Y0 rgb = f_d, then f_v). */
void orc_decode_sh(int64_t n, const double *h, const orc_sh_mlp *mlp_d,
                   const orc_sh_mlp *mlp_v, double *Y);

/* Value of an IEEE binary16 bit pattern. */
double orc_half_to_double(uint16_t b);

/* Round to the nearest bfloat16 value, ties to even. */
double orc_bf16_round(double v);

/* Eq. 4 on one feature vector x[22]: out = (phi, o, d_r, d_g, d_b), with BF16
 * rounding applied to x, h1 and h2 (the tensor-core inputs). */
void orc_mlp_eval(const orc_mlp *mlp, const double x[22], double out[5]);

/* Preprocess all n Gaussians.  attrs: n x 24 values (stored precision,
 * widened exactly).  Returns 0 on success. */
int orc_preprocess(int64_t n, const double *attrs, const orc_camera *cam,
                   const orc_mlp *mlp, int use_mlp, int rgb_residual,
                   orc_gauss *out);

/* Tile lists (ascending Gaussian index within each tile).  offsets has
 * tiles_x * tiles_y + 1 entries.  gids may be NULL to only count.  Returns the
 * number of (tile, Gaussian) pairs K, or -1 if K > cap. */
int64_t orc_bin(int64_t n, const orc_gauss *g, int tiles_x, int tiles_y,
                int64_t *offsets, int32_t *gids, int64_t cap);

/* FP32-contract tile test of binning: 1 if Gaussian g may include a pixel
 * centre of tile (tx, ty) (conservative slab bounds at the tile centre), 0 if
 * it certainly includes none.  The tile lists hold the visible Gaussians whose
 * rectangle contains the tile and that pass this test. */
int orc_tile_may_hit(const orc_gauss *g, int tx, int ty);

/* FP32-contract inclusion test of pixel (px, py) for Gaussian g. */
int orc_includes(const orc_gauss *g, int px, int py);

/* Eq. 2 over the tiles [tile_begin, tile_end) (row-major tile index).
 * out_rgb: H x W x 3.  out_aux (optional): 5 x H x W planes
 * (A_r, A_g, A_b, B, T) with A = sum c a w, B = sum a w, T = prod (1 - a).
 * out_count (optional): H x W number of included Gaussians. */
/* Rendered depth for the depth distillation of Sec. 3.2 (Eq. 5): the
 * depth-aware weighted mean of the included Gaussians' view depths,
 * D = sum d a w / sum a w (0 where nothing is included), with the same
 * inclusion test, alpha and weights as Eq. 2.  out_depth: H x W. */
int orc_rasterize_depth(int64_t n, const orc_gauss *g, const int64_t *offsets,
                        const int32_t *gids, int width, int height,
                        int tile_begin, int tile_end, double *out_depth);

int orc_rasterize(int64_t n, const orc_gauss *g, const int64_t *offsets,
                  const int32_t *gids, int width, int height,
                  const double bg[3], int tile_begin, int tile_end,
                  double *out_rgb, double *out_aux, int32_t *out_count);

/* Sorted front-to-back alpha blending (App. B, Eq. 11: C = sum c_i a_i T_i,
 * T_i = prod_{j<i} (1 - a_j)), the 3DGS compositing the paper replaces; kept
 * as the comparator of the sort-free renderer.  Per pixel the included
 * Gaussians are ordered by FP32-contract view depth (ties by index); blending
 * stops before the Gaussian that would bring T below 1e-4 (3DGS early
 * termination); C += T c_bg at the end.  out_count (optional): Gaussians
 * blended per pixel. */
int orc_rasterize_sorted(int64_t n, const orc_gauss *g, const int64_t *offsets,
                         const int32_t *gids, int width, int height,
                         const double bg[3], int tile_begin, int tile_end,
                         double *out_rgb, int32_t *out_count);

/* All included (pixel, Gaussian) pairs: pixel index py * width + px and
 * Gaussian index, tile by tile, pixel by pixel, list order.  Returns the
 * number of pairs, or -1 if it exceeds cap (outputs may be NULL to count). */
int64_t orc_pairs(const orc_gauss *g, const int64_t *offsets, const int32_t *gids,
                  int width, int height, int64_t *out_pixel, int32_t *out_gid,
                  int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
