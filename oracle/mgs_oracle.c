/*
 * FP64 CPU oracle for the Mobile-GS sort-free renderer.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product renderer.  Plain,
 * single-threaded, unblocked loops that follow the paper's equations in the
 * paper's order.  Build with -ffp-contract=off (the FP32 contract below needs
 * every binary32 operation rounded exactly as written).
 *
 * Paper passages followed:
 *   App. B   3D Gaussians (mu, Sigma = R S S^T R^T, o, Y) and their
 *            perspective projection (3DGS convention, inherited).
 *   Sec. 3.1 Eq. 2  C = (1 - T) sum(c_i a_i w_i) / sum(a_i w_i) + T c_bg,
 *                   T = prod(1 - a_j), a_i = o_i exp(-1/2 dx^T Sigma^-1 dx).
 *   Sec. 3.1 Eq. 3  w_i = phi_i^2 + phi_i / d_i^2 + exp(s_max / d_i).
 *   Sec. 3.1 Eq. 4  F = MLP_f(P_i, s_i, r_i, Y_i); phi = ReLU(MLP_phi F);
 *                   o = sigmoid(MLP_o F); P_i = (mu_i - t_v)/|mu_i - t_v|.
 *   Sec. 3.2        first-order SH (3 x 4 coefficients) colour.
 *   Sec. 2, Eq. 1 discussion: sums commute, so any accumulation order is valid.
 *
 * Readings where the paper is silent (3DGS conventions): near plane 0.2,
 * frustum clamp 1.3 * tan(fov/2) in the EWA Jacobian, 0.3 px^2 dilation of
 * Sigma_2D, radius ceil(3 sqrt(lambda_max)), inclusion q <= 9, alpha clamped
 * to 0.99, SH colour offset +0.5 then max(0, .), d = view-space z,
 * s_max = largest activated scale, phi = 1 without the MLP, foreground term 0
 * when sum(a w) = 0.
 */
#include "mgs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

int64_t orc_gauss_size(void) { return (int64_t)sizeof(orc_gauss); }

/* ------------------------------------------------------------------------- */
/* Plain FP64 helpers                                                         */
/* ------------------------------------------------------------------------- */

/* Unit quaternion (w, x, y, z) -> rotation matrix, row-major (textbook). */
void orc_rotation(const double q[4], double R[9])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Nearest bfloat16 (8 significant bits), ties to even. */
double orc_bf16_round(double v)
{
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    double m = frexp(v, &e);              /* v = m 2^e, 0.5 <= |m| < 1 */
    double r = nearbyint(ldexp(m, 8));     /* default mode: ties to even */
    return ldexp(r, e - 8);
}

static double bf16_bits_to_double(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

/* Eq. 4.  MLP_f = two ReLU layers (22 -> 64 -> 64); MLP_phi and MLP_o (and the
 * optional colour residual) are the rows of one linear head (64 -> 5).  The
 * tensor-core inputs (x, h1, h2) are rounded to BF16; everything else FP64. */
/* One hidden layer: out = BF16(ReLU(W in + b)), in and W as given. */
static void hidden_layer(const uint16_t *w, const float *b, const double *in, int n_in,
                         int n_out, double *out)
{
    for (int j = 0; j < n_out; ++j) {
        double acc = 0.0;
        for (int i = 0; i < n_in; ++i)
            acc += bf16_bits_to_double(w[j * n_in + i]) * in[i];
        acc += (double)b[j];
        out[j] = orc_bf16_round(acc > 0.0 ? acc : 0.0);
    }
}

void orc_mlp_eval(const orc_mlp *mlp, const double x[22], double out[5])
{
    /* Eq. 4 with BF16 inputs to every layer: F = MLP_f([P, s, q, Y]), then the
     * phi and o heads (and the optional colour residual rows). */
    double xr[22], ha[256], hb[256];
    for (int i = 0; i < 22; ++i) xr[i] = orc_bf16_round(x[i]);
    const uint16_t *wh;
    const float *bh;
    int nh;
    const double *last;
    if (mlp->h1 == 0) {
        hidden_layer(mlp->w1, mlp->b1, xr, 22, 64, ha);
        hidden_layer(mlp->w2, mlp->b2, ha, 64, 64, hb);
        wh = mlp->w3; bh = mlp->b3; nh = 64; last = hb;
    } else {
        hidden_layer(mlp->w1, mlp->b1, xr, 22, mlp->h1, ha);
        hidden_layer(mlp->w2, mlp->b2, ha, mlp->h1, mlp->h2, hb);
        hidden_layer(mlp->w3, mlp->b3, hb, mlp->h2, mlp->h3, ha);
        wh = mlp->w4; bh = mlp->b4; nh = mlp->h3; last = ha;
    }
    double y[5];
    for (int k = 0; k < 5; ++k) {
        double acc = 0.0;
        for (int i = 0; i < nh; ++i)
            acc += bf16_bits_to_double(wh[k * nh + i]) * last[i];
        y[k] = acc + (double)bh[k];
    }
    out[0] = y[0] > 0.0 ? y[0] : 0.0;          /* phi = ReLU(MLP_phi F) */
    out[1] = 1.0 / (1.0 + exp(-y[1]));         /* o = sigmoid(MLP_o F)  */
    out[2] = y[2];
    out[3] = y[3];
    out[4] = y[4];
}

/* ------------------------------------------------------------------------- */
/* FP32 contract: visibility, tile rectangle, inclusion predicate             */
/* ------------------------------------------------------------------------- */
/*
 * Every line below is one correctly rounded binary32 operation (or an fmaf,
 * rounded once).  The same sequence, evaluated by any IEEE-754 machine,
 * yields bit-identical rectangles and predicate factors.  Returns 1 if the
 * Gaussian is visible.
 */
static int contract_f32(const double *a, const orc_camera *cam, int tiles_x,
                        int tiles_y, int32_t rect[4], float m[2], float l[3],
                        float *depth)
{
    const float mux = (float)a[0], muy = (float)a[1], muz = (float)a[2];
    const float s[3] = {(float)a[3], (float)a[4], (float)a[5]};
    const float qw = (float)a[6], qx = (float)a[7], qy = (float)a[8],
                qz = (float)a[9];
    const float *W = cam->R;

    /* normalised quaternion and its rotation matrix */
    float n2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    if (!(n2 > 0.0f)) return 0;
    float qn = sqrtf(n2);
    float w = qw / qn, x = qx / qn, y = qy / qn, z = qz / qn;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz);
    R[1] = 2.0f * (xy - wz);
    R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz);
    R[4] = 1.0f - 2.0f * (xx + zz);
    R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy);
    R[7] = 2.0f * (yz + wx);
    R[8] = 1.0f - 2.0f * (xx + yy);

    /* camera-space mean, near-plane cull */
    float tx = fmaf(W[0], mux, fmaf(W[1], muy, fmaf(W[2], muz, cam->t[0])));
    float ty = fmaf(W[3], mux, fmaf(W[4], muy, fmaf(W[5], muz, cam->t[1])));
    float tz = fmaf(W[6], mux, fmaf(W[7], muy, fmaf(W[8], muz, cam->t[2])));
    *depth = tz;
    if (!(tz > cam->znear)) return 0;

    /* EWA Jacobian with the frustum clamp */
    float rz = 1.0f / tz;
    float txz = tx * rz, tyz = ty * rz;
    float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
    float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
    float txc = fminf(fmaxf(txz, -limx), limx);
    float tyc = fminf(fmaxf(tyz, -limy), limy);
    float J00 = cam->fx * rz, J02 = -((cam->fx * txc) * rz);
    float J11 = cam->fy * rz, J12 = -((cam->fy * tyc) * rz);

    /* T = J W (2x3), M = R(q) diag(s), V = T M, Sigma_2D = V V^T + 0.3 I */
    float T0[3], T1[3], M[9], V0[3], V1[3];
    for (int j = 0; j < 3; ++j) {
        T0[j] = fmaf(J02, W[6 + j], J00 * W[j]);
        T1[j] = fmaf(J12, W[6 + j], J11 * W[3 + j]);
    }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) M[3 * k + j] = R[3 * k + j] * s[j];
    for (int j = 0; j < 3; ++j) {
        V0[j] = fmaf(T0[2], M[6 + j], fmaf(T0[1], M[3 + j], T0[0] * M[j]));
        V1[j] = fmaf(T1[2], M[6 + j], fmaf(T1[1], M[3 + j], T1[0] * M[j]));
    }
    float ca = fmaf(V0[0], V0[0], fmaf(V0[1], V0[1], V0[2] * V0[2])) + 0.3f;
    float cb = fmaf(V0[0], V1[0], fmaf(V0[1], V1[1], V0[2] * V1[2]));
    float cc = fmaf(V1[0], V1[0], fmaf(V1[1], V1[1], V1[2] * V1[2])) + 0.3f;
    float det = fmaf(ca, cc, -(cb * cb));
    if (!(det > 0.0f)) return 0;

    /* pixel mean */
    float mx = fmaf(cam->fx, txz, cam->cx);
    float my = fmaf(cam->fy, tyz, cam->cy);

    /* radius from the largest eigenvalue, tile rectangle */
    float mid = 0.5f * (ca + cc);
    float hd = 0.5f * (ca - cc);
    float lam = mid + sqrtf(fmaf(hd, hd, cb * cb));
    float rad = ceilf(3.0f * sqrtf(lam));
    float v[4];
    v[0] = floorf((mx - rad) * 0.0625f);
    v[1] = floorf((my - rad) * 0.0625f);
    v[2] = floorf((mx + rad) * 0.0625f) + 1.0f;
    v[3] = floorf((my + rad) * 0.0625f) + 1.0f;
    const float lim[4] = {(float)tiles_x, (float)tiles_y, (float)tiles_x,
                          (float)tiles_y};
    for (int i = 0; i < 4; ++i) {
        float c = v[i] > 0.0f ? v[i] : 0.0f;
        c = c < lim[i] ? c : lim[i];
        rect[i] = (int32_t)c;
    }
    if (rect[0] >= rect[2] || rect[1] >= rect[3]) return 0;

    /* predicate factors: Sigma_2D^-1 = L L^T with
       l11 = sqrt(c / det), l21 = -b / sqrt(c det), l22 = 1 / sqrt(c) */
    l[0] = sqrtf(cc / det);
    l[1] = -(cb / sqrtf(cc * det));
    l[2] = 1.0f / sqrtf(cc);
    m[0] = mx;
    m[1] = my;
    return 1;
}

/* Inclusion: q = (l11 dx + l21 dy)^2 + (l22 dy)^2 <= 9, dx = x + 0.5 - m_x. */
int orc_includes(const orc_gauss *g, int px, int py)
{
    float dx = ((float)px + 0.5f) - g->m32[0];
    float dy = ((float)py + 0.5f) - g->m32[1];
    float e1 = fmaf(g->l32[0], dx, g->l32[1] * dy);
    float e2 = g->l32[2] * dy;
    float q = fmaf(e1, e1, e2 * e2);
    return q <= 9.0f;
}

/* ------------------------------------------------------------------------- */
/* Preprocess (App. B projection, Sec. 3.2 colour, Eq. 3, Eq. 4)              */
/* ------------------------------------------------------------------------- */

static const double SH_C0 = 0.28209479177387814;  /* 1 / (2 sqrt(pi))       */
static const double SH_C1 = 0.4886025119029199;   /* sqrt(3) / (2 sqrt(pi)) */

int orc_preprocess(int64_t n, const double *attrs, const orc_camera *cam,
                   const orc_mlp *mlp, int use_mlp, int rgb_residual,
                   orc_gauss *out)
{
    if (use_mlp && !mlp) return -1;
    const int tiles_x = (cam->width + ORC_TILE - 1) / ORC_TILE;
    const int tiles_y = (cam->height + ORC_TILE - 1) / ORC_TILE;
    double W[9], tc[3];
    for (int i = 0; i < 9; ++i) W[i] = (double)cam->R[i];
    for (int i = 0; i < 3; ++i) tc[i] = (double)cam->t[i];
    const double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy;
    /* camera centre t_v = -W^T t */
    double cc[3];
    for (int j = 0; j < 3; ++j)
        cc[j] = -(W[j] * tc[0] + W[3 + j] * tc[1] + W[6 + j] * tc[2]);

    for (int64_t i = 0; i < n; ++i) {
        const double *a = attrs + i * ORC_REC;
        orc_gauss *g = out + i;
        memset(g, 0, sizeof *g);
        g->visible = contract_f32(a, cam, tiles_x, tiles_y, g->rect, g->m32,
                                  g->l32, &g->tz32);

        const double mu[3] = {a[0], a[1], a[2]};
        const double s[3] = {a[3], a[4], a[5]};
        double qn = sqrt(a[6] * a[6] + a[7] * a[7] + a[8] * a[8] + a[9] * a[9]);
        double qh[4] = {a[6] / qn, a[7] / qn, a[8] / qn, a[9] / qn};
        double R[9];
        orc_rotation(qh, R);

        /* camera space */
        double t[3];
        for (int r = 0; r < 3; ++r)
            t[r] = W[3 * r] * mu[0] + W[3 * r + 1] * mu[1] + W[3 * r + 2] * mu[2] +
                   tc[r];
        g->depth = t[2];

        /* Sigma_3D = R S S^T R^T */
        double S3[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[3 * r + k] * s[k] * s[k] * R[3 * c + k];
                S3[3 * r + c] = acc;
            }
        /* camera-space covariance W Sigma_3D W^T */
        double SC[9], tmp[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += W[3 * r + k] * S3[3 * k + c];
                tmp[3 * r + c] = acc;
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += tmp[3 * r + k] * W[3 * c + k];
                SC[3 * r + c] = acc;
            }
        /* Jacobian of the perspective projection at the (clamped) mean */
        double limx = 1.3 * (0.5 * cam->width / fx);
        double limy = 1.3 * (0.5 * cam->height / fy);
        double txz = t[0] / t[2], tyz = t[1] / t[2];
        double txc = txz < -limx ? -limx : (txz > limx ? limx : txz);
        double tyc = tyz < -limy ? -limy : (tyz > limy ? limy : tyz);
        double J[6] = {fx / t[2], 0.0, -fx * txc / t[2],
                       0.0, fy / t[2], -fy * tyc / t[2]};
        double JS[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * SC[3 * k + c];
                JS[3 * r + c] = acc;
            }
        double S2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += JS[3 * r + k] * J[3 * c + k];
                S2[2 * r + c] = acc;
            }
        double ca = S2[0] + 0.3, cb = 0.5 * (S2[1] + S2[2]), ccv = S2[3] + 0.3;
        double det = ca * ccv - cb * cb;
        g->cov[0] = ca;
        g->cov[1] = cb;
        g->cov[2] = ccv;
        g->conic[0] = ccv / det;
        g->conic[1] = -cb / det;
        g->conic[2] = ca / det;
        g->mean[0] = fx * txz + cx;
        g->mean[1] = fy * tyz + cy;

        /* viewing direction P_i (Sec. 3.1) */
        double d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) g->dir[k] = d[k] / dn;

        /* phi and o (Eq. 4, or phi = 1 and the stored opacity) */
        double res[5] = {1.0, a[10], 0.0, 0.0, 0.0};
        if (use_mlp) {
            double x[22];
            for (int k = 0; k < 3; ++k) x[k] = g->dir[k];
            for (int k = 0; k < 3; ++k) x[3 + k] = s[k];
            for (int k = 0; k < 4; ++k) x[6 + k] = qh[k];
            for (int k = 0; k < 12; ++k) x[10 + k] = a[11 + k];
            orc_mlp_eval(mlp, x, res);
        }
        g->phi = res[0];
        g->opacity = res[1];

        /* degree-1 SH colour (Sec. 3.2), 3DGS basis signs */
        const double Px = g->dir[0], Py = g->dir[1], Pz = g->dir[2];
        for (int ch = 0; ch < 3; ++ch) {
            double v = SH_C0 * a[11 + ch] - SH_C1 * Py * a[14 + ch] +
                       SH_C1 * Pz * a[17 + ch] - SH_C1 * Px * a[20 + ch] + 0.5;
            if (use_mlp && rgb_residual) v += res[2 + ch];
            g->rgb[ch] = v > 0.0 ? v : 0.0;
        }

        /* Eq. 3 */
        double smax = s[0] > s[1] ? s[0] : s[1];
        smax = smax > s[2] ? smax : s[2];
        double phi = g->phi, dd = g->depth;
        g->weight = phi * phi + phi / (dd * dd) + exp(smax / dd);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tile binning: per-tile Gaussian lists, no depth order                      */
/* ------------------------------------------------------------------------- */

/* FP32 contract, binning: can Gaussian g include any pixel centre of tile
 * (tx, ty)?  Slab bounds at the tile centre (bx, by) with half extent 7.5:
 * every pixel p of the tile has |e1(p)| >= |e1c| - h1 and |e2(p)| >=
 * |e2c| - h2 (exact arithmetic), and an included pixel has |e1|, |e2| <= 3;
 * the margins m1, m2 (2^-18 relative) cover the rounding of both sides, so a
 * tile that fails holds no included pixel.  One correctly rounded binary32
 * operation per line, as the GPU evaluates it. */
int orc_tile_may_hit(const orc_gauss *g, int tx, int ty)
{
    const float mx = g->m32[0], my = g->m32[1];
    const float l11 = g->l32[0], l21 = g->l32[1], l22 = g->l32[2];
    const float bx = (float)(tx * ORC_TILE + 8), by = (float)(ty * ORC_TILE + 8);
    const float h = 7.5f;
    const float dxb = bx - mx;
    const float dyb = by - my;
    const float t21 = l21 * dyb;
    const float e1c = fabsf(fmaf(l11, dxb, t21));
    const float a21 = fabsf(l21) * h;
    const float h1 = fmaf(fabsf(l11), h, a21);
    const float u1 = fabsf(dxb) + h;
    const float u2 = fabsf(dyb) + h;
    const float s11 = fabsf(l11) * u1;
    const float s12 = fabsf(l21) * u2;
    const float s1 = s11 + s12;
    const float s1b = s1 + 4.0f;
    const float m1 = 3.814697265625e-06f * s1b;
    const float e2c = fabsf(l22 * dyb);
    const float h2 = fabsf(l22) * h;
    const float s2 = fabsf(l22) * u2;
    const float s2b = s2 + 4.0f;
    const float m2 = 3.814697265625e-06f * s2b;
    const float d1 = e1c - h1, d2 = e2c - h2;
    const float c1 = 3.0f + m1, c2 = 3.0f + m2;
    return d1 <= c1 && d2 <= c2;
}

int64_t orc_bin(int64_t n, const orc_gauss *g, int tiles_x, int tiles_y,
                int64_t *offsets, int32_t *gids, int64_t cap)
{
    const int64_t T = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t <= T; ++t) offsets[t] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!g[i].visible) continue;
        for (int ty = g[i].rect[1]; ty < g[i].rect[3]; ++ty)
            for (int tx = g[i].rect[0]; tx < g[i].rect[2]; ++tx)
                if (orc_tile_may_hit(g + i, tx, ty)) offsets[(int64_t)ty * tiles_x + tx + 1] += 1;
    }
    for (int64_t t = 0; t < T; ++t) offsets[t + 1] += offsets[t];
    const int64_t K = offsets[T];
    if (!gids) return K;
    if (K > cap) return -1;
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
    if (!cur) return -1;
    for (int64_t t = 0; t < T; ++t) cur[t] = offsets[t];
    for (int64_t i = 0; i < n; ++i) {
        if (!g[i].visible) continue;
        for (int ty = g[i].rect[1]; ty < g[i].rect[3]; ++ty)
            for (int tx = g[i].rect[0]; tx < g[i].rect[2]; ++tx)
                if (orc_tile_may_hit(g + i, tx, ty)) gids[cur[(int64_t)ty * tiles_x + tx]++] = (int32_t)i;
    }
    free(cur);
    return K;
}

/* ------------------------------------------------------------------------- */
/* Eq. 2: per-pixel normalised, depth-weighted composite                      */
/* ------------------------------------------------------------------------- */

int orc_rasterize(int64_t n, const orc_gauss *g, const int64_t *offsets,
                  const int32_t *gids, int width, int height,
                  const double bg[3], int tile_begin, int tile_end,
                  double *out_rgb, double *out_aux, int32_t *out_count)
{
    (void)n;
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    const int64_t HW = (int64_t)width * height;
    for (int t = tile_begin; t < tile_end; ++t) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < height; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < width; ++px) {
                double A[3] = {0.0, 0.0, 0.0}, B = 0.0, T = 1.0;
                int32_t cnt = 0;
                for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k) {
                    const orc_gauss *gi = g + gids[k];
                    if (!orc_includes(gi, px, py)) continue;
                    double dx = px + 0.5 - gi->mean[0];
                    double dy = py + 0.5 - gi->mean[1];
                    double q = gi->conic[0] * dx * dx + 2.0 * gi->conic[1] * dx * dy +
                               gi->conic[2] * dy * dy;
                    double alpha = gi->opacity * exp(-0.5 * q);
                    if (alpha > 0.99) alpha = 0.99;
                    double aw = alpha * gi->weight;
                    for (int ch = 0; ch < 3; ++ch) A[ch] += gi->rgb[ch] * aw;
                    B += aw;
                    T *= 1.0 - alpha;
                    cnt += 1;
                }
                const int64_t p = (int64_t)py * width + px;
                for (int ch = 0; ch < 3; ++ch) {
                    double fg = B > 0.0 ? (1.0 - T) * A[ch] / B : 0.0;
                    out_rgb[3 * p + ch] = fg + T * bg[ch];
                }
                if (out_aux) {
                    for (int ch = 0; ch < 3; ++ch) out_aux[ch * HW + p] = A[ch];
                    out_aux[3 * HW + p] = B;
                    out_aux[4 * HW + p] = T;
                }
                if (out_count) out_count[p] = cnt;
            }
    }
    return 0;
}

/* Sec. 3.2, Eq. 5 reading: the depth image the distillation loss compares is
 * the depth-aware weighted mean depth, D = sum_i d_i a_i w_i / sum_i a_i w_i,
 * over the Gaussians included at the pixel (Eq. 2's weights a_i w_i). */
int orc_rasterize_depth(int64_t n, const orc_gauss *g, const int64_t *offsets,
                        const int32_t *gids, int width, int height,
                        int tile_begin, int tile_end, double *out_depth)
{
    (void)n;
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    for (int t = tile_begin; t < tile_end; ++t) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < height; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < width; ++px) {
                double Ad = 0.0, B = 0.0;
                for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k) {
                    const orc_gauss *gi = g + gids[k];
                    if (!orc_includes(gi, px, py)) continue;
                    double dx = px + 0.5 - gi->mean[0];
                    double dy = py + 0.5 - gi->mean[1];
                    double q = gi->conic[0] * dx * dx + 2.0 * gi->conic[1] * dx * dy +
                               gi->conic[2] * dy * dy;
                    double alpha = gi->opacity * exp(-0.5 * q);
                    if (alpha > 0.99) alpha = 0.99;
                    double aw = alpha * gi->weight;
                    Ad += gi->depth * aw;
                    B += aw;
                }
                out_depth[(int64_t)py * width + px] = B > 0.0 ? Ad / B : 0.0;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Included pairs (for the differentiable FP64 restatement in grad.py)         */
/* ------------------------------------------------------------------------- */

int64_t orc_pairs(const orc_gauss *g, const int64_t *offsets, const int32_t *gids,
                  int width, int height, int64_t *out_pixel, int32_t *out_gid,
                  int64_t cap)
{
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    const int tiles_y = (height + ORC_TILE - 1) / ORC_TILE;
    int64_t k = 0;
    for (int t = 0; t < tiles_x * tiles_y; ++t) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < height; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < width; ++px)
                for (int64_t j = offsets[t]; j < offsets[t + 1]; ++j) {
                    if (!orc_includes(g + gids[j], px, py)) continue;
                    if (out_pixel && out_gid) {
                        if (k >= cap) return -1;
                        out_pixel[k] = (int64_t)py * width + px;
                        out_gid[k] = gids[j];
                    }
                    ++k;
                }
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Comparator: sorted front-to-back alpha blending (App. B, Eq. 11)            */
/* ------------------------------------------------------------------------- */

static const orc_gauss *g_sort_base;

static int by_depth(const void *x, const void *y)
{
    const int32_t i = *(const int32_t *)x, j = *(const int32_t *)y;
    const float di = g_sort_base[i].tz32, dj = g_sort_base[j].tz32;
    if (di < dj) return -1;
    if (di > dj) return 1;
    return (i > j) - (i < j);
}

int orc_rasterize_sorted(int64_t n, const orc_gauss *g, const int64_t *offsets,
                         const int32_t *gids, int width, int height,
                         const double bg[3], int tile_begin, int tile_end,
                         double *out_rgb, int32_t *out_count)
{
    (void)n;
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    int64_t maxlen = 1;
    for (int t = tile_begin; t < tile_end; ++t)
        if (offsets[t + 1] - offsets[t] > maxlen) maxlen = offsets[t + 1] - offsets[t];
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)maxlen);
    if (!list) return -1;
    g_sort_base = g;
    for (int t = tile_begin; t < tile_end; ++t) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < height; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < width; ++px) {
                int64_t m = 0;
                for (int64_t k = offsets[t]; k < offsets[t + 1]; ++k)
                    if (orc_includes(g + gids[k], px, py)) list[m++] = gids[k];
                qsort(list, (size_t)m, sizeof(int32_t), by_depth);
                double C[3] = {0.0, 0.0, 0.0}, T = 1.0;
                int32_t cnt = 0;
                for (int64_t k = 0; k < m; ++k) {
                    const orc_gauss *gi = g + list[k];
                    double dx = px + 0.5 - gi->mean[0];
                    double dy = py + 0.5 - gi->mean[1];
                    double q = gi->conic[0] * dx * dx + 2.0 * gi->conic[1] * dx * dy +
                               gi->conic[2] * dy * dy;
                    double alpha = gi->opacity * exp(-0.5 * q);
                    if (alpha > 0.99) alpha = 0.99;
                    double next = T * (1.0 - alpha);
                    if (next < 1e-4) break;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += gi->rgb[ch] * alpha * T;
                    T = next;
                    cnt += 1;
                }
                const int64_t p = (int64_t)py * width + px;
                for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = C[ch] + T * bg[ch];
                if (out_count) out_count[p] = cnt;
            }
    }
    free(list);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2, Eq. 6: SH features decoded once at load time                     */
/* ------------------------------------------------------------------------- */

/* IEEE binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
double orc_half_to_double(uint16_t b)
{
    const int sign = (b >> 15) & 1, e = (b >> 10) & 31, f = b & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);                 /* subnormal: f * 2^-14 / 2^10 */
    else if (e == 31)
        v = f ? NAN : INFINITY;
    else
        v = ldexp(1.0 + f / 1024.0, e - 15);
    return sign ? -v : v;
}

static void sh_mlp_eval(const orc_sh_mlp *m, const double in[6], double *out)
{
    double hid[64];
    for (int j = 0; j < 64; ++j) {
        double acc = orc_half_to_double(m->b1[j]);
        for (int i = 0; i < 6; ++i) acc += orc_half_to_double(m->w1[j * 6 + i]) * in[i];
        hid[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int k = 0; k < m->n_out; ++k) {
        double acc = orc_half_to_double(m->b2[k]);
        for (int j = 0; j < 64; ++j) acc += orc_half_to_double(m->w2[k * 64 + j]) * hid[j];
        out[k] = acc;
    }
}

void orc_decode_sh(int64_t n, const double *h, const orc_sh_mlp *mlp_d,
                   const orc_sh_mlp *mlp_v, double *Y)
{
    for (int64_t i = 0; i < n; ++i) {
        sh_mlp_eval(mlp_d, h + 6 * i, Y + 12 * i);       /* f_d -> Y0 rgb */
        sh_mlp_eval(mlp_v, h + 6 * i, Y + 12 * i + 3);   /* f_v -> Y1..Y3 rgb */
    }
}
