/*
 * darb_oracle.c -- plain CPU oracle of the DARB-Splatting rasterizer.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark call this code; the product path never does.
 * It shares no source with the CUDA library.
 *
 * What it computes (paper Sec. 4, Eq. darbf_class, Eq. 2x2covProjection,
 * Table 1, Table 2 and the listings of supplementary Sec. B):
 *   - per splat: the projected mean mu', the psi-corrected, dilated 2D
 *     covariance Sigma2 and its inverse (the conic), the 3-sigma radius, the
 *     pixel-exact tile rectangle, view depth and the SH colour;
 *   - per pixel p: the front-to-back alpha composite, in ascending depth, of
 *     alpha_i(p) = min(0.99, o_i F_k(q_i(p))), q = (p - mu')^T Sigma2^-1 (p - mu'),
 *     with F_k truncated to its main lobe (Sec. A.3), the 3DGS thresholds
 *     (skip alpha < 1/255, stop before T(1 - alpha) < 1e-4) and background;
 *   - the analytic FP64 gradient of that composite w.r.t. every input.
 *
 * Two numeric tracks.  Everything that turns floating point into a discrete
 * decision (culling, radius, tile rectangle, depth order, the q cutoff) is
 * evaluated by a fixed IEEE FP32 operation sequence ("geom32", the paper's
 * FP32 rasterizer) or, for finite-difference checks, by the same formulas in
 * FP64 ("geom64").  Kernel values, alpha, transmittance and colour are FP64.
 * The alpha and transmittance thresholds are taken in FP64; when one lies
 * within a stated margin of its threshold, both branches are followed and
 * every resulting outcome is reported (several results are then correct).
 *
 * Render modes: brute force (every non-culled splat, explicitly depth sorted,
 * tested at every pixel; the splat counts at a pixel only if the pixel's tile
 * lies in the splat's tile rectangle) and tiled (per-tile lists built by an
 * explicit sort of (tile, depth, id)).  The two give identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    float viewmat[16]; /* world -> camera, row-major, OpenCV axes */
    float fx, fy, cx, cy, near_plane;
    int width, height;
    float bg[3];
} orc_camera;

typedef struct {
    int kind;
    float psi;
    float q_max;
    int q_max_strict;
    /* kind K_GENERIC only: Table 1's "modified" family F = base(u), u = d_M^beta / xi */
    int base;
    float xi, beta;
    int lobes;
} orc_kernel;

typedef struct {
    int culled, radius, rect[4], tiles, clampx, clampy;
    float depth;
    double mean2d[2], conic[3];
} orc_proj;

typedef struct {
    int pixel, count, last_id, primary;
    double T, C[3];
    uint64_t sig;
} orc_outcome;

enum { K_GAUSSIAN = 0, K_HALF_COSINE, K_RAISED_COSINE, K_MOD_SINC, K_INV_QUADRIC,
       K_INV_MULTIQUADRIC, K_PARABOLA, K_GENERIC, K_COUNT };

/* 3DGS compositing constants, as FP32 literals. */
#define ALPHA_MAX ((double)0.99f)
#define ALPHA_MIN ((double)(1.0f / 255.0f))
#define T_MIN ((double)0.0001f)

/* ------------------------------------------------------------------------ */
/* Projection, in FP32 and FP64 (one body, two instantiations).             */

#define REAL float
#define FMA fmaf
#define SQRT sqrtf
#define CEIL ceilf
#define FLOOR floorf
#define FMIN fminf
#define FMAX fmaxf
#define PROJECT_FN project_f32
#include "project_impl.h"
#undef REAL
#undef FMA
#undef SQRT
#undef CEIL
#undef FLOOR
#undef FMIN
#undef FMAX
#undef PROJECT_FN

#define REAL double
#define FMA fma
#define SQRT sqrt
#define CEIL ceil
#define FLOOR floor
#define FMIN fmin
#define FMAX fmax
#define PROJECT_FN project_f64
#include "project_impl.h"
#undef REAL
#undef FMA
#undef SQRT
#undef CEIL
#undef FLOOR
#undef FMIN
#undef FMAX
#undef PROJECT_FN

/* ------------------------------------------------------------------------ */
/* Kernel profiles F(q), q = d_M^2 (Table 1 with the xi of Table 2, read in */
/* the forms the Sec. B listings evaluate).                                 */

/* Table 1's modified members, F = base(u) with u = d_M^beta / xi = q^(beta/2) / xi:
 * base 0 exp(-u), 1 cos(u), 2 1/2 + 1/2 cos(u), 3 |sin u| / u, 4 (u + 1)^(-1/2), 5 1 - u. */
static double generic_u(const orc_kernel *k, double q)
{
    if (q <= 0.0) return 0.0;
    return pow(q, 0.5 * (double)k->beta) / (double)k->xi;
}

static double generic_base(int base, double u)
{
    switch (base) {
    case 0: return exp(-u);
    case 1: return cos(u);
    case 2: return 0.5 + 0.5 * cos(u);
    case 3: return u == 0.0 ? 1.0 : fabs(sin(u)) / u;
    case 4: return 1.0 / sqrt(u + 1.0);
    case 5: return 1.0 - u;
    }
    return 0.0;
}

static double generic_base_du(int base, double u)
{
    switch (base) {
    case 0: return -exp(-u);
    case 1: return -sin(u);
    case 2: return -0.5 * sin(u);
    case 3: {
        if (u < 1e-3) return -u / 3.0 + u * u * u / 30.0; /* series of (u cos u - sin u) / u^2 */
        const double sg = sin(u) < 0.0 ? -1.0 : 1.0;
        return sg * (u * cos(u) - sin(u)) / (u * u);
    }
    case 4: return -0.5 * pow(u + 1.0, -1.5);
    case 5: return -1.0;
    }
    return 0.0;
}

/* dF/dq = dF/du (beta/2) u / q; at q = 0 the one-sided limit is evaluated at q = 1e-24 (finite
 * for beta = 2; for beta < 2 it diverges unless dF/du vanishes at u = 0). */
static double generic_dq(const orc_kernel *k, double q)
{
    const double hb = 0.5 * (double)k->beta;
    if (hb == 1.0) return generic_base_du(k->base, q / (double)k->xi) / (double)k->xi;
    const double qq = q > 1e-24 ? q : 1e-24;
    const double u = pow(qq, hb) / (double)k->xi;
    return generic_base_du(k->base, u) * hb * u / qq;
}

static double F_value_k(const orc_kernel *k, double q);
static double F_deriv_k(const orc_kernel *k, double q);

static double F_value(int kind, double q)
{
    switch (kind) {
    case K_GAUSSIAN: /* exp(-d^2 / xi), xi = 2 */
        return exp(-0.5 * q);
    case K_HALF_COSINE: /* cos(d^2 / xi), xi = 18/pi  (Eq. HalfCosine) */
        return cos(M_PI * q / 18.0);
    case K_RAISED_COSINE: /* 0.5 + 0.5 cos(d / xi), xi = 2.5/pi  (Sec. B.1) */
        return 0.5 + 0.5 * cos(M_PI * sqrt(q) / 2.5);
    case K_MOD_SINC: { /* |sin(d/xi)| / (d/xi), xi = 3/pi  (Sec. B.3); F(0) = 1 */
        const double x = M_PI * sqrt(q) / 3.0;
        return x == 0.0 ? 1.0 : fabs(sin(x)) / x;
    }
    case K_INV_QUADRIC: /* 1 / (d^2 + 1)  (Sec. B.4 listing) */
        return 1.0 / (1.0 + q);
    case K_INV_MULTIQUADRIC: /* 1 / sqrt(d^2 / xi + 1), xi = 1  (Table 1) */
        return 1.0 / sqrt(1.0 + q);
    case K_PARABOLA: /* 1 - d^2 / xi, xi = 9  (Table 1, Sec. B.5) */
        return 1.0 - q / 9.0;
    }
    return 0.0;
}

/* dF/dq.  Near q = 0 the raised cosine and the sinc use their Taylor series
 * (the closed forms are 0/0 there); the limits are the continuous extension. */
static double F_deriv(int kind, double q)
{
    switch (kind) {
    case K_GAUSSIAN:
        return -0.5 * exp(-0.5 * q);
    case K_HALF_COSINE:
        return -(M_PI / 18.0) * sin(M_PI * q / 18.0);
    case K_RAISED_COSINE: {
        const double k = M_PI / 2.5;
        if (q < 1e-12) return -k * k / 4.0 + k * k * k * k * q / 24.0;
        const double r = sqrt(q);
        return -(k / 4.0) * sin(k * r) / r;
    }
    case K_MOD_SINC: {
        const double x = M_PI * sqrt(q) / 3.0;
        if (x < 0.1) { /* F = sum (-1)^n x^(2n)/(2n+1)!, x^2 = a q */
            const double a = M_PI * M_PI / 9.0;
            return -a / 6.0 + a * a * q / 60.0 - a * a * a * q * q / 1680.0 +
                   a * a * a * a * q * q * q / 90720.0;
        }
        return (x * cos(x) - sin(x)) / (2.0 * q * x);
    }
    case K_INV_QUADRIC:
        return -1.0 / ((1.0 + q) * (1.0 + q));
    case K_INV_MULTIQUADRIC:
        return -0.5 * pow(1.0 + q, -1.5);
    case K_PARABOLA:
        return -1.0 / 9.0;
    }
    return 0.0;
}

static double F_value_k(const orc_kernel *k, double q)
{
    return k->kind == K_GENERIC ? generic_base(k->base, generic_u(k, q)) : F_value(k->kind, q);
}

static double F_deriv_k(const orc_kernel *k, double q)
{
    return k->kind == K_GENERIC ? generic_dq(k, q) : F_deriv(k->kind, q);
}

void orc_kernel_eval(int kind, int n, const double *q, double *F, double *dF)
{
    for (int i = 0; i < n; ++i) {
        if (F) F[i] = F_value(kind, q[i]);
        if (dF) dF[i] = F_deriv(kind, q[i]);
    }
}

/* F and dF/dq of any kernel, the generic family included. */
void orc_kernel_eval_k(const orc_kernel *k, int n, const double *q, double *F, double *dF)
{
    for (int i = 0; i < n; ++i) {
        if (F) F[i] = F_value_k(k, q[i]);
        if (dF) dF[i] = F_deriv_k(k, q[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics to degree 3 (3DGS ordering m = -l..l, with the  */
/* Condon-Shortley phase), normalisation constants from their closed forms. */

static void sh_basis(int deg, double x, double y, double z, double *Y, double (*dY)[3])
{
    const double sp = sqrt(M_PI);
    const double c0 = 1.0 / (2.0 * sp);
    const double c1 = sqrt(3.0) / (2.0 * sp);
    const double c2a = sqrt(15.0) / (2.0 * sp); /* xy, yz, xz terms */
    const double c2b = sqrt(5.0) / (4.0 * sp);  /* 2z^2 - x^2 - y^2 */
    const double c2c = sqrt(15.0) / (4.0 * sp); /* x^2 - y^2 */
    const double c3a = sqrt(35.0 / (2.0 * M_PI)) / 4.0;
    const double c3b = sqrt(105.0 / M_PI) / 2.0;
    const double c3c = sqrt(21.0 / (2.0 * M_PI)) / 4.0;
    const double c3d = sqrt(7.0 / M_PI) / 4.0;
    const double c3e = sqrt(105.0 / M_PI) / 4.0;
    const int K = (deg + 1) * (deg + 1);
    double g[16][3];
    memset(g, 0, sizeof g);
    Y[0] = c0;
    if (deg >= 1) {
        Y[1] = -c1 * y; g[1][1] = -c1;
        Y[2] = c1 * z;  g[2][2] = c1;
        Y[3] = -c1 * x; g[3][0] = -c1;
    }
    if (deg >= 2) {
        const double xx = x * x, yy = y * y, zz = z * z;
        Y[4] = c2a * x * y;                 g[4][0] = c2a * y; g[4][1] = c2a * x;
        Y[5] = -c2a * y * z;                g[5][1] = -c2a * z; g[5][2] = -c2a * y;
        Y[6] = c2b * (2 * zz - xx - yy);    g[6][0] = -2 * c2b * x; g[6][1] = -2 * c2b * y; g[6][2] = 4 * c2b * z;
        Y[7] = -c2a * x * z;                g[7][0] = -c2a * z; g[7][2] = -c2a * x;
        Y[8] = c2c * (xx - yy);             g[8][0] = 2 * c2c * x; g[8][1] = -2 * c2c * y;
    }
    if (deg >= 3) {
        const double xx = x * x, yy = y * y, zz = z * z;
        Y[9] = -c3a * y * (3 * xx - yy);
        g[9][0] = -c3a * 6 * x * y; g[9][1] = -c3a * (3 * xx - 3 * yy);
        Y[10] = c3b * x * y * z;
        g[10][0] = c3b * y * z; g[10][1] = c3b * x * z; g[10][2] = c3b * x * y;
        Y[11] = -c3c * y * (4 * zz - xx - yy);
        g[11][0] = c3c * 2 * x * y; g[11][1] = -c3c * (4 * zz - xx - 3 * yy); g[11][2] = -c3c * 8 * y * z;
        Y[12] = c3d * z * (2 * zz - 3 * xx - 3 * yy);
        g[12][0] = -c3d * 6 * x * z; g[12][1] = -c3d * 6 * y * z; g[12][2] = c3d * (6 * zz - 3 * xx - 3 * yy);
        Y[13] = -c3c * x * (4 * zz - xx - yy);
        g[13][0] = -c3c * (4 * zz - 3 * xx - yy); g[13][1] = c3c * 2 * x * y; g[13][2] = -c3c * 8 * x * z;
        Y[14] = c3e * z * (xx - yy);
        g[14][0] = c3e * 2 * x * z; g[14][1] = -c3e * 2 * y * z; g[14][2] = c3e * (xx - yy);
        Y[15] = -c3a * x * (xx - 3 * yy);
        g[15][0] = -c3a * (3 * xx - 3 * yy); g[15][1] = c3a * 6 * x * y;
    }
    if (dY)
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < 3; ++j) dY[k][j] = g[k][j];
}

void orc_sh_basis(int deg, int n, const double *dirs, double *Y, double *dY)
{
    const int K = (deg + 1) * (deg + 1);
    for (int i = 0; i < n; ++i) {
        double g[16][3];
        sh_basis(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Y + (size_t)K * i, g);
        if (dY)
            for (int k = 0; k < K; ++k)
                for (int j = 0; j < 3; ++j) dY[((size_t)K * i + k) * 3 + j] = g[k][j];
    }
}

static void camera_centre(const orc_camera *cam, double c[3])
{
    /* viewmat = [R t; 0 1]  =>  centre = -R^T t */
    for (int j = 0; j < 3; ++j) {
        c[j] = 0.0;
        for (int r = 0; r < 3; ++r) c[j] -= (double)cam->viewmat[4 * r + j] * (double)cam->viewmat[4 * r + 3];
    }
}

/* ------------------------------------------------------------------------ */
/* Tile membership.  A splat's tiles are, row of tiles by row of tiles, those */
/* whose pixel columns meet the x-extent of its ellipse {q <= q_max} over    */
/* the row's band of pixel-centre heights: the extent's ends are the         */
/* ellipse's leftmost and rightmost points, clamped to the band, so every    */
/* pixel centre with q <= q_max lies in a member tile.  Tiles of the row     */
/* form one run [c0, c1] inside the rectangle.  The FP32 track takes the     */
/* fixed IEEE sequence below (the GPU takes the same one), the FP64 track    */
/* the same formulas in double.                                              */

/* Per splat: det, the extents and 1/A; per row: the band, the heights of the ellipse's         */
/* rightmost and leftmost points clamped to it, the x offsets there and the run.  At the        */
/* unclamped heights dyR0 = -B xm / C and -dyR0 the offsets are exactly xm and -xm (substitute  */
/* dyR0 into the root), and are taken as such.                                                  */
#define SPAN_BODY(R, SQ, CE, FL, MX, MN)                                                      \
    const R det = A * C - B * B;                                                             \
    if (!(det > (R)0)) return 0;                                                             \
    const R xm = SQ((qm * C) / det), ym = SQ((qm * A) / det);                                \
    const R nB = -B;                                                                         \
    const R dyR0 = (nB * xm) / C, dyL0 = -dyR0;                                              \
    const R aq = A * qm;                                                                     \
    const R invA = (R)1 / A;                                                                 \
    const R ya = (R)(ty * tile) + (R)0.5f;                                                   \
    const R yb = MN((R)(ty * tile + tile) - (R)0.5f, (R)H - (R)0.5f);                       \
    const R ea = MX(ya - u1, -ym), eb = MN(yb - u1, ym);                                     \
    if (!(ea <= eb)) return 0;                                                               \
    const R dyR = MN(MX(dyR0, ea), eb), dyL = MN(MX(dyL0, ea), eb);                         \
    const R right = dyR == dyR0 ? xm : (nB * dyR + SQ(MX(aq - det * (dyR * dyR), (R)0))) * invA; \
    const R left = dyL == dyL0 ? -xm : (nB * dyL - SQ(MX(aq - det * (dyL * dyL), (R)0))) * invA; \
    const R i0 = MX(CE((u0 + left) - (R)0.5f), (R)0);                                        \
    const R i1 = MN(FL((u0 + right) - (R)0.5f), (R)(W - 1));                                \
    if (!(i0 <= i1)) return 0;                                                               \
    int a0 = (int)i0 / tile, a1 = (int)i1 / tile;                                            \
    if (a0 < r[0]) a0 = r[0];                                                                \
    if (a1 > r[2]) a1 = r[2];                                                                \
    if (a0 > a1) return 0;                                                                   \
    *c0 = a0;                                                                                \
    *c1 = a1;                                                                                \
    return 1;

static int span_f32(float u0, float u1, float A, float B, float C, float qm, int tile, int W, int H,
                    const int *r, int ty, int *c0, int *c1)
{
    SPAN_BODY(float, sqrtf, ceilf, floorf, fmaxf, fminf)
}

static int span_f64(double u0, double u1, double A, double B, double C, double qm, int tile, int W, int H,
                    const int *r, int ty, int *c0, int *c1)
{
    SPAN_BODY(double, sqrt, ceil, floor, fmax, fmin)
}

/* The run of member tiles of splat i in tile row ty; 0 if none. */
static int row_span(int geom32, const double *mean2d, const double *conic, int i, float qmax, int tile, int W,
                    int H, const int *rect, int ty, int *c0, int *c1)
{
    const int *r = rect + 4 * (size_t)i;
    if (ty < r[1] || ty > r[3]) return 0;
    const double *m = mean2d + 2 * (size_t)i, *k = conic + 3 * (size_t)i;
    if (geom32)
        return span_f32((float)m[0], (float)m[1], (float)k[0], (float)k[1], (float)k[2], qmax, tile, W, H, r, ty,
                        c0, c1);
    return span_f64(m[0], m[1], k[0], k[1], k[2], (double)qmax, tile, W, H, r, ty, c0, c1);
}

static int span_count(int geom32, const double *mean2d, const double *conic, int i, float qmax, int tile, int W,
                      int H, const int *rect)
{
    int n = 0, c0, c1;
    for (int ty = rect[4 * (size_t)i + 1]; ty <= rect[4 * (size_t)i + 3]; ++ty)
        if (row_span(geom32, mean2d, conic, i, qmax, tile, W, H, rect, ty, &c0, &c1)) n += c1 - c0 + 1;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Per-splat preprocessing.                                                 */

int orc_project(int n, const float *means, const float *scales, const float *quats,
                const float *sh, int sh_degree, const orc_camera *cam, const orc_kernel *k,
                int tile, int geom32,
                int *culled, int *radius, int *rect, int *tiles, float *depth, int *clampxy,
                double *mean2d, double *conic, double *rgb, unsigned char *clamped)
{
    if (n < 0 || sh_degree < 0 || sh_degree > 3 || tile <= 0) return 1;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    double cc[3];
    camera_centre(cam, cc);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        orc_proj p;
        if (geom32)
            project_f32(means + 3 * (size_t)i, scales + 3 * (size_t)i, quats + 4 * (size_t)i, cam, k->psi, tile, &p);
        else
            project_f64(means + 3 * (size_t)i, scales + 3 * (size_t)i, quats + 4 * (size_t)i, cam, k->psi, tile, &p);
        culled[i] = p.culled;
        radius[i] = p.culled ? 0 : p.radius;
        for (int j = 0; j < 4; ++j) rect[4 * (size_t)i + j] = p.rect[j];
        tiles[i] = 0;
        depth[i] = p.depth;
        clampxy[2 * (size_t)i] = p.clampx;
        clampxy[2 * (size_t)i + 1] = p.clampy;
        mean2d[2 * (size_t)i] = p.mean2d[0];
        mean2d[2 * (size_t)i + 1] = p.mean2d[1];
        for (int j = 0; j < 3; ++j) conic[3 * (size_t)i + j] = p.conic[j];
        /* SH colour, FP64: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5) */
        double d[3], len = 0.0;
        for (int j = 0; j < 3; ++j) {
            d[j] = (double)means[3 * (size_t)i + j] - cc[j];
            len += d[j] * d[j];
        }
        len = sqrt(len);
        double Y[16];
        sh_basis(sh_degree, d[0] / len, d[1] / len, d[2] / len, Y, NULL);
        unsigned char cl = 0;
        for (int ch = 0; ch < 3; ++ch) {
            double v = 0.0;
            for (int kk = 0; kk < K; ++kk) v += Y[kk] * (double)sh[((size_t)i * K + kk) * 3 + ch];
            v += 0.5;
            if (v < 0.0) {
                v = 0.0;
                cl |= (unsigned char)(1u << ch);
            }
            rgb[3 * (size_t)i + ch] = v;
        }
        clamped[i] = cl;
        if (!p.culled) { /* a splat whose ellipse reaches no tile is culled, like an empty rectangle */
            tiles[i] = span_count(geom32, mean2d, conic, i, k->q_max, tile, cam->width, cam->height, rect);
            if (tiles[i] == 0) {
                culled[i] = 1;
                radius[i] = 0;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tile lists: one instance per (splat, tile in its rectangle), sorted by   */
/* (tile, depth, splat id).  Depth is positive, so its IEEE bits order like */
/* the value; key = tile << 32 | bits(depth).                               */

typedef struct {
    uint64_t key;
    int id;
} instance;

static int cmp_instance(const void *pa, const void *pb)
{
    const instance *a = (const instance *)pa, *b = (const instance *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

static uint32_t float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

long long orc_build_lists(int n, const int *culled, const int *rect, const float *depth, const double *mean2d,
                          const double *conic, float qmax, int geom32, int tile, int width, int height,
                          int tiles_x, int tiles_y, const unsigned char *tile_mask,
                          uint64_t *keys, int *ids, long long capacity, int *ranges)
{
    long long M = 0;
    int c0, c1;
    for (int i = 0; i < n; ++i) {
        if (culled[i]) continue;
        const int *r = rect + 4 * (size_t)i;
        for (int ty = r[1]; ty <= r[3]; ++ty) {
            if (!row_span(geom32, mean2d, conic, i, qmax, tile, width, height, rect, ty, &c0, &c1)) continue;
            for (int tx = c0; tx <= c1; ++tx)
                if (!tile_mask || tile_mask[ty * tiles_x + tx]) ++M;
        }
    }
    if (!keys) return M;
    if (M > capacity) return -1;
    instance *inst = (instance *)malloc(sizeof(instance) * (size_t)(M > 0 ? M : 1));
    if (!inst) return -2;
    long long m = 0;
    for (int i = 0; i < n; ++i) {
        if (culled[i]) continue;
        const int *r = rect + 4 * (size_t)i;
        for (int ty = r[1]; ty <= r[3]; ++ty) {
            if (!row_span(geom32, mean2d, conic, i, qmax, tile, width, height, rect, ty, &c0, &c1)) continue;
            for (int tx = c0; tx <= c1; ++tx) {
                const int t = ty * tiles_x + tx;
                if (tile_mask && !tile_mask[t]) continue;
                inst[m].key = ((uint64_t)t << 32) | float_bits(depth[i]);
                inst[m].id = i;
                ++m;
            }
        }
    }
    qsort(inst, (size_t)M, sizeof(instance), cmp_instance);
    for (int t = 0; t < tiles_x * tiles_y; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (long long j = 0; j < M; ++j) {
        keys[j] = inst[j].key;
        ids[j] = inst[j].id;
        const int t = (int)(inst[j].key >> 32);
        if (j == 0 || (int)(inst[j - 1].key >> 32) != t) ranges[2 * t] = (int)j;
        ranges[2 * t + 1] = (int)(j + 1);
    }
    free(inst);
    return M;
}

/* ------------------------------------------------------------------------ */
/* The per-pixel walk.                                                      */

typedef struct {
    const int *rect;
    const double *mean2d, *conic, *rgb;
    const float *opac;
    int geom32, kind, strict;
    float qmax;
    orc_kernel kp;
    const int *seq;
    int len;
    int tx, ty;
    int check_member, tile, W, H; /* brute force: test the splat's tile membership per pixel */
    float px, py;
    double bg[3];
    double eps_a, eps_t;
    orc_outcome *outs;
    int nout, cap, unverifiable;
} walk_ctx;

typedef struct {
    int count, last_id;
    double T, C[3];
    uint64_t sig;
} walk_state;

/* Support test and alpha of splat id at this pixel; 0 if it does not apply. */
static int eval_alpha(const walk_ctx *c, int id, double *alpha, double *F, double *q)
{
    if (c->check_member) { /* tiled lists hold members only */
        int c0, c1;
        if (!row_span(c->geom32, c->mean2d, c->conic, id, c->qmax, c->tile, c->W, c->H, c->rect, c->ty, &c0, &c1) ||
            c->tx < c0 || c->tx > c1)
            return 0;
    }
    double qq;
    if (c->geom32) { /* q by the fixed FP32 sequence: q = dx (A dx + 2B dy) + (C dy) dy */
        const float mx = (float)c->mean2d[2 * (size_t)id], my = (float)c->mean2d[2 * (size_t)id + 1];
        const float A = (float)c->conic[3 * (size_t)id], B = (float)c->conic[3 * (size_t)id + 1],
                    C = (float)c->conic[3 * (size_t)id + 2];
        const float dx = mx - c->px, dy = my - c->py;
        const float e = (2.0f * B) * dy;
        const float g = fmaf(A, dx, e);
        const float h = (C * dy) * dy;
        const float qf = fmaf(dx, g, h);
        if (qf < 0.0f || (c->strict ? qf >= c->qmax : qf > c->qmax)) return 0;
        qq = (double)qf;
    } else {
        const double dx = c->mean2d[2 * (size_t)id] - (double)c->px;
        const double dy = c->mean2d[2 * (size_t)id + 1] - (double)c->py;
        const double A = c->conic[3 * (size_t)id], B = c->conic[3 * (size_t)id + 1], C = c->conic[3 * (size_t)id + 2];
        qq = fma(dx, fma(A, dx, (2.0 * B) * dy), (C * dy) * dy);
        if (qq < 0.0 || (c->strict ? qq >= (double)c->qmax : qq > (double)c->qmax)) return 0;
    }
    const double Fv = F_value_k(&c->kp, qq);
    double a = (double)c->opac[id] * Fv;
    if (a > ALPHA_MAX) a = ALPHA_MAX;
    *alpha = a;
    *F = Fv;
    *q = qq;
    return 1;
}

enum { D_SKIP = 0, D_STOP = 1, D_BLEND = 2 };

static void record(walk_ctx *c, const walk_state *s, int primary)
{
    if (c->nout >= c->cap) {
        c->unverifiable = 1;
        return;
    }
    orc_outcome *o = &c->outs[c->nout++];
    o->count = s->count;
    o->last_id = s->last_id;
    o->primary = primary;
    o->T = s->T;
    for (int ch = 0; ch < 3; ++ch) o->C[ch] = s->C[ch] + s->T * c->bg[ch];
    o->sig = s->sig;
}

static void blend(const walk_ctx *c, walk_state *s, int id, double a, double tn)
{
    for (int ch = 0; ch < 3; ++ch) s->C[ch] += c->rgb[3 * (size_t)id + ch] * a * s->T;
    s->T = tn;
    s->count += 1;
    s->last_id = id;
    s->sig = s->sig * 1000003ull ^ (uint64_t)(id + 1);
}

static void walk(walk_ctx *c, int pos, walk_state s, int budget, int primary)
{
    for (; pos < c->len; ++pos) {
        const int id = c->seq[pos];
        double a, F, q;
        if (!eval_alpha(c, id, &a, &F, &q)) continue;
        const double tn = s.T * (1.0 - a);
        const int skip64 = a < ALPHA_MIN;
        const int amb_a = fabs(a - ALPHA_MIN) <= c->eps_a;
        const int stop64 = tn < T_MIN;
        const int amb_t = fabs(tn - T_MIN) <= c->eps_t * T_MIN;
        const int kind64 = skip64 ? D_SKIP : (stop64 ? D_STOP : D_BLEND);
        int possible[3] = {0, 0, 0};
        for (int ia = 0; ia < 2; ++ia) {
            if (ia && !amb_a) continue;
            const int sk = ia ? !skip64 : skip64;
            if (sk) {
                possible[D_SKIP] = 1;
                continue;
            }
            for (int it = 0; it < 2; ++it) {
                if (it && !amb_t) continue;
                const int st = it ? !stop64 : stop64;
                possible[st ? D_STOP : D_BLEND] = 1;
            }
        }
        for (int kd = 0; kd < 3; ++kd) {
            if (!possible[kd] || kd == kind64) continue;
            if (budget <= 0) {
                c->unverifiable = 1;
                continue;
            }
            walk_state s2 = s;
            if (kd == D_STOP) record(c, &s2, 0);
            else {
                if (kd == D_BLEND) blend(c, &s2, id, a, tn);
                walk(c, pos + 1, s2, budget - 1, 0);
            }
        }
        if (kind64 == D_STOP) {
            record(c, &s, primary);
            return;
        }
        if (kind64 == D_BLEND) blend(c, &s, id, a, tn);
    }
    record(c, &s, primary);
}

static void init_ctx(walk_ctx *c, const int *rect, const double *mean2d, const double *conic,
                     const float *opac, const double *rgb, int geom32, const orc_camera *cam,
                     const orc_kernel *k, double eps_a, double eps_t)
{
    memset(c, 0, sizeof *c);
    c->rect = rect;
    c->mean2d = mean2d;
    c->conic = conic;
    c->opac = opac;
    c->rgb = rgb;
    c->geom32 = geom32;
    c->kind = k->kind;
    c->kp = *k;
    c->qmax = k->q_max;
    c->strict = k->q_max_strict;
    for (int ch = 0; ch < 3; ++ch) c->bg[ch] = cam->bg[ch];
    c->eps_a = eps_a;
    c->eps_t = eps_t;
}

typedef struct {
    float depth;
    int id;
} depth_id;

static int cmp_depth_id(const void *pa, const void *pb)
{
    const depth_id *a = (const depth_id *)pa, *b = (const depth_id *)pb;
    const uint32_t ua = float_bits(a->depth), ub = float_bits(b->depth);
    if (ua != ub) return ua < ub ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

#define MAX_OUT 32

/* mode 0: brute force over all splats; mode 1: tiled lists (ids, ranges).
 * Pixels of tiles not in tile_mask (when given) are left untouched. */
int orc_render(int n, const int *culled, const int *rect, const float *depth,
               const double *mean2d, const double *conic, const float *opac, const double *rgb,
               int geom32, const orc_camera *cam, const orc_kernel *k, int tile, int mode,
               const int *ids, const int *ranges, const unsigned char *tile_mask,
               double eps_alpha, double eps_T, int max_branch,
               double *image, double *T_final, int *count, int *last_id, int *amb, uint64_t *sig,
               orc_outcome *alts, int alts_cap, int *n_alts)
{
    const int W = cam->width, H = cam->height;
    const int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
    int *order = NULL;
    int norder = 0;
    if (mode == 0) {
        depth_id *di = (depth_id *)malloc(sizeof(depth_id) * (size_t)(n > 0 ? n : 1));
        order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
        if (!di || !order) return 2;
        for (int i = 0; i < n; ++i)
            if (!culled[i]) {
                di[norder].depth = depth[i];
                di[norder].id = i;
                ++norder;
            }
        qsort(di, (size_t)norder, sizeof(depth_id), cmp_depth_id);
        for (int j = 0; j < norder; ++j) order[j] = di[j].id;
        free(di);
    }
    int nalts = 0;
    const int ntiles = tiles_x * tiles_y;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < ntiles; ++t) {
        if (tile_mask && !tile_mask[t]) continue;
        const int tx = t % tiles_x, ty = t / tiles_x;
        orc_outcome outs[MAX_OUT];
        walk_ctx c;
        init_ctx(&c, rect, mean2d, conic, opac, rgb, geom32, cam, k, eps_alpha, eps_T);
        c.outs = outs;
        c.cap = MAX_OUT;
        c.tx = tx;
        c.ty = ty;
        c.check_member = mode == 0;
        c.tile = tile;
        c.W = W;
        c.H = H;
        if (mode == 0) {
            c.seq = order;
            c.len = norder;
        } else {
            c.seq = ids + ranges[2 * t];
            c.len = ranges[2 * t + 1] - ranges[2 * t];
        }
        for (int py = ty * tile; py < (ty + 1) * tile && py < H; ++py)
            for (int px = tx * tile; px < (tx + 1) * tile && px < W; ++px) {
                const int pix = py * W + px;
                c.px = (float)px + 0.5f;
                c.py = (float)py + 0.5f;
                c.nout = 0;
                c.unverifiable = 0;
                walk_state s;
                memset(&s, 0, sizeof s);
                s.T = 1.0;
                s.last_id = -1;
                walk(&c, 0, s, max_branch, 1);
                int prim = 0;
                for (int j = 0; j < c.nout; ++j)
                    if (outs[j].primary) prim = j;
                for (int ch = 0; ch < 3; ++ch) image[(size_t)ch * W * H + pix] = outs[prim].C[ch];
                T_final[pix] = outs[prim].T;
                count[pix] = outs[prim].count;
                last_id[pix] = outs[prim].last_id;
                sig[pix] = outs[prim].sig;
                amb[pix] = c.unverifiable ? 2 : (c.nout > 1 ? 1 : 0);
                if (alts && c.nout > 1)
                    for (int j = 0; j < c.nout; ++j) {
                        if (j == prim) continue;
                        int slot;
#pragma omp atomic capture
                        slot = nalts++;
                        if (slot < alts_cap) {
                            alts[slot] = outs[j];
                            alts[slot].pixel = pix;
                        }
                    }
            }
    }
    free(order);
    if (n_alts) *n_alts = nalts;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward of the composite (tiled lists, FP64 decisions).                 */
/* grad2d per splat: d mu'x, d mu'y, dA, dB, dC (conic q = A dx^2 + 2B dx dy */
/* + C dy^2), d opacity, d r, d g, d b.                                     */

int orc_render_backward(int n, const int *rect, const double *mean2d, const double *conic,
                        const float *opac, const double *rgb, int geom32, const orc_camera *cam,
                        const orc_kernel *k, int tile, const int *ids, const int *ranges,
                        long long M, const unsigned char *tile_mask, const double *dL_dimage,
                        double *grad2d)
{
    const int W = cam->width, H = cam->height;
    const int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
    const int ntiles = tiles_x * tiles_y;
    double *contrib = (double *)calloc((size_t)(M > 0 ? M : 1) * 9, sizeof(double));
    if (!contrib) return 2;
    int maxlen = 0;
    for (int t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    int err = 0;
#pragma omp parallel
    {
        int *bpos = (int *)malloc(sizeof(int) * (size_t)(maxlen + 1));
        double *ba = (double *)malloc(sizeof(double) * (size_t)(maxlen + 1) * 4);
        if (!bpos || !ba) {
#pragma omp atomic write
            err = 2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < ntiles; ++t) {
            if (!bpos || !ba) continue;
            if (tile_mask && !tile_mask[t]) continue;
            const int tx = t % tiles_x, ty = t / tiles_x;
            const int start = ranges[2 * t], len = ranges[2 * t + 1] - ranges[2 * t];
            walk_ctx c;
            init_ctx(&c, rect, mean2d, conic, opac, rgb, geom32, cam, k, 0.0, 0.0);
            c.tx = tx;
            c.ty = ty;
            for (int py = ty * tile; py < (ty + 1) * tile && py < H; ++py)
                for (int px = tx * tile; px < (tx + 1) * tile && px < W; ++px) {
                    const int pix = py * W + px;
                    const double g[3] = {dL_dimage[pix], dL_dimage[(size_t)W * H + pix],
                                         dL_dimage[2 * (size_t)W * H + pix]};
                    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
                    c.px = (float)px + 0.5f;
                    c.py = (float)py + 0.5f;
                    /* forward walk with FP64 decisions, keeping the blended list */
                    int nb = 0;
                    double T = 1.0;
                    for (int pos = 0; pos < len; ++pos) {
                        const int id = ids[start + pos];
                        double a, F, q;
                        if (!eval_alpha(&c, id, &a, &F, &q)) continue;
                        if (a < ALPHA_MIN) continue;
                        const double tn = T * (1.0 - a);
                        if (tn < T_MIN) break;
                        bpos[nb] = pos;
                        ba[4 * nb + 0] = a;
                        ba[4 * nb + 1] = F;
                        ba[4 * nb + 2] = q;
                        ba[4 * nb + 3] = T;
                        ++nb;
                        T = tn;
                    }
                    /* S = everything composited behind the current splat */
                    double S[3];
                    for (int ch = 0; ch < 3; ++ch) S[ch] = T * c.bg[ch];
                    for (int j = nb - 1; j >= 0; --j) {
                        const int pos = bpos[j], id = ids[start + pos];
                        const double a = ba[4 * j], F = ba[4 * j + 1], q = ba[4 * j + 2], Tk = ba[4 * j + 3];
                        const double *col = rgb + 3 * (size_t)id;
                        double *out = contrib + 9 * (size_t)(start + pos);
                        double dalpha = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            dalpha += g[ch] * (col[ch] * Tk - S[ch] / (1.0 - a));
                            out[6 + ch] += a * Tk * g[ch];
                        }
                        for (int ch = 0; ch < 3; ++ch) S[ch] += col[ch] * a * Tk;
                        const double o = (double)opac[id];
                        if (o * F > ALPHA_MAX) continue; /* clamped: alpha is constant */
                        out[5] += F * dalpha;
                        const double dq = o * F_deriv_k(k, q) * dalpha;
                        const double dx = mean2d[2 * (size_t)id] - (double)c.px;
                        const double dy = mean2d[2 * (size_t)id + 1] - (double)c.py;
                        const double A = conic[3 * (size_t)id], B = conic[3 * (size_t)id + 1],
                                     C = conic[3 * (size_t)id + 2];
                        out[0] += dq * 2.0 * (A * dx + B * dy);
                        out[1] += dq * 2.0 * (B * dx + C * dy);
                        out[2] += dq * dx * dx;
                        out[3] += dq * 2.0 * dx * dy;
                        out[4] += dq * dy * dy;
                    }
                }
        }
        free(bpos);
        free(ba);
    }
    if (err) {
        free(contrib);
        return err;
    }
    memset(grad2d, 0, sizeof(double) * 9 * (size_t)n);
    for (long long j = 0; j < M; ++j) {
        const int id = ids[j];
        for (int v = 0; v < 9; ++v) grad2d[9 * (size_t)id + v] += contrib[9 * (size_t)j + v];
    }
    free(contrib);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward of the per-splat preprocessing, FP64 chain rule.                */

static void backward_splat(const float *mi, const float *si, const float *qi, const float *shi,
                           int deg, const orc_camera *cam, double psi, int clampx, int clampy,
                           unsigned char clampedrgb, const double *cc, const double *g,
                           double *dm, double *ds, double *dq, double *dsh)
{
    double V[16];
    for (int j = 0; j < 16; ++j) V[j] = cam->viewmat[j];
    const double m[3] = {mi[0], mi[1], mi[2]};
    double t[3];
    for (int r = 0; r < 3; ++r) t[r] = V[4 * r] * m[0] + V[4 * r + 1] * m[1] + V[4 * r + 2] * m[2] + V[4 * r + 3];
    const double tx = t[0], ty = t[1], tz = t[2];

    /* rotation from the normalised quaternion */
    const double qv[4] = {qi[0], qi[1], qi[2], qi[3]};
    const double qn = sqrt(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
    const double w = qv[0] / qn, x = qv[1] / qn, y = qv[2] / qn, z = qv[3] / qn;
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    const double s[3] = {si[0], si[1], si[2]};
    double M[3][3], Sig[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) M[j][l] = R[j][l] * s[l];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) Sig[j][l] = M[j][0] * M[l][0] + M[j][1] * M[l][1] + M[j][2] * M[l][2];

    /* Jacobian (guard-band clamp decided by the forward) */
    const double fx = cam->fx, fy = cam->fy;
    const double limx = (double)1.3f * ((double)cam->width / (2.0 * fx));
    const double limy = (double)1.3f * ((double)cam->height / (2.0 * fy));
    const double txtz = tx / tz, tytz = ty / tz;
    const double Lx = txtz < 0 ? -limx : limx, Ly = tytz < 0 ? -limy : limy;
    const double txc = clampx ? Lx * tz : tx, tyc = clampy ? Ly * tz : ty;
    const double J00 = fx / tz, J02 = -fx * txc / (tz * tz), J11 = fy / tz, J12 = -fy * tyc / (tz * tz);
    double Tm[2][3];
    for (int kk = 0; kk < 3; ++kk) {
        Tm[0][kk] = J00 * V[kk] + J02 * V[8 + kk];
        Tm[1][kk] = J11 * V[4 + kk] + J12 * V[8 + kk];
    }
    double TS[2][3], s2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int kk = 0; kk < 3; ++kk) TS[r][kk] = Tm[r][0] * Sig[0][kk] + Tm[r][1] * Sig[1][kk] + Tm[r][2] * Sig[2][kk];
    for (int r = 0; r < 2; ++r)
        for (int l = 0; l < 2; ++l) s2[r][l] = TS[r][0] * Tm[l][0] + TS[r][1] * Tm[l][1] + TS[r][2] * Tm[l][2];
    const double a = psi * s2[0][0] + (double)0.3f, b = psi * s2[0][1], c = psi * s2[1][1] + (double)0.3f;
    const double det = a * c - b * b;
    const double K[2][2] = {{c / det, -b / det}, {-b / det, a / det}};

    /* conic -> Sigma2: dSigma2 = -K G K, G the symmetric conic gradient */
    const double G[2][2] = {{g[2], 0.5 * g[3]}, {0.5 * g[3], g[4]}};
    double KG[2][2], dS2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int l = 0; l < 2; ++l) KG[r][l] = K[r][0] * G[0][l] + K[r][1] * G[1][l];
    for (int r = 0; r < 2; ++r)
        for (int l = 0; l < 2; ++l) dS2[r][l] = -(KG[r][0] * K[0][l] + KG[r][1] * K[1][l]);
    /* Sigma2 = psi Sigma' + 0.3 I */
    double dsp[2][2];
    for (int r = 0; r < 2; ++r)
        for (int l = 0; l < 2; ++l) dsp[r][l] = psi * dS2[r][l];
    /* Sigma' = Tm Sig Tm^T: dSig = Tm^T dsp Tm, dTm = 2 dsp Tm Sig */
    double dSig[3][3], dTm[2][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            double v = 0.0;
            for (int r = 0; r < 2; ++r)
                for (int u = 0; u < 2; ++u) v += Tm[r][j] * dsp[r][u] * Tm[u][l];
            dSig[j][l] = v;
        }
    for (int r = 0; r < 2; ++r)
        for (int kk = 0; kk < 3; ++kk) dTm[r][kk] = 2.0 * (dsp[r][0] * TS[0][kk] + dsp[r][1] * TS[1][kk]);
    /* Tm = J W: dJ_rj = sum_k dTm_rk W_jk */
    double dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
    for (int kk = 0; kk < 3; ++kk) {
        dJ00 += dTm[0][kk] * V[kk];
        dJ02 += dTm[0][kk] * V[8 + kk];
        dJ11 += dTm[1][kk] * V[4 + kk];
        dJ12 += dTm[1][kk] * V[8 + kk];
    }
    double dt[3] = {0.0, 0.0, 0.0};
    const double tz2 = tz * tz, tz3 = tz2 * tz;
    dt[2] += dJ00 * (-fx / tz2) + dJ11 * (-fy / tz2);
    if (!clampx) {
        dt[0] += dJ02 * (-fx / tz2);
        dt[2] += dJ02 * (2.0 * fx * tx / tz3);
    } else
        dt[2] += dJ02 * (fx * Lx / tz2);
    if (!clampy) {
        dt[1] += dJ12 * (-fy / tz2);
        dt[2] += dJ12 * (2.0 * fy * ty / tz3);
    } else
        dt[2] += dJ12 * (fy * Ly / tz2);
    /* projected mean: u = f t_xy / t_z + c */
    dt[0] += g[0] * fx / tz;
    dt[1] += g[1] * fy / tz;
    dt[2] += -g[0] * fx * tx / tz2 - g[1] * fy * ty / tz2;
    for (int j = 0; j < 3; ++j) dm[j] = V[j] * dt[0] + V[4 + j] * dt[1] + V[8 + j] * dt[2];

    /* Sigma = M M^T: dM = 2 dSig M; M = R diag(s) */
    double dM[3][3], dR[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) dM[j][l] = 2.0 * (dSig[j][0] * M[0][l] + dSig[j][1] * M[1][l] + dSig[j][2] * M[2][l]);
    for (int l = 0; l < 3; ++l) {
        ds[l] = dM[0][l] * R[0][l] + dM[1][l] * R[1][l] + dM[2][l] * R[2][l];
        for (int j = 0; j < 3; ++j) dR[j][l] = dM[j][l] * s[l];
    }
    /* R(w, x, y, z) */
    const double Rw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
    const double Rx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
    const double Ry[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
    const double Rz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
    double dn[4] = {0, 0, 0, 0};
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            dn[0] += dR[j][l] * Rw[j][l];
            dn[1] += dR[j][l] * Rx[j][l];
            dn[2] += dR[j][l] * Ry[j][l];
            dn[3] += dR[j][l] * Rz[j][l];
        }
    /* normalisation q -> q/|q| */
    const double nv[4] = {w, x, y, z};
    const double ndot = nv[0] * dn[0] + nv[1] * dn[1] + nv[2] * dn[2] + nv[3] * dn[3];
    for (int j = 0; j < 4; ++j) dq[j] = (dn[j] - nv[j] * ndot) / qn;

    /* SH colour */
    const int Kc = (deg + 1) * (deg + 1);
    double v[3], len = 0.0;
    for (int j = 0; j < 3; ++j) {
        v[j] = m[j] - cc[j];
        len += v[j] * v[j];
    }
    len = sqrt(len);
    const double dir[3] = {v[0] / len, v[1] / len, v[2] / len};
    double Y[16], dY[16][3];
    sh_basis(deg, dir[0], dir[1], dir[2], Y, dY);
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        const double gr = (clampedrgb >> ch) & 1 ? 0.0 : g[6 + ch];
        for (int kk = 0; kk < Kc; ++kk) {
            dsh[kk * 3 + ch] = Y[kk] * gr;
            for (int j = 0; j < 3; ++j) ddir[j] += gr * (double)shi[kk * 3 + ch] * dY[kk][j];
        }
    }
    const double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
    for (int j = 0; j < 3; ++j) dm[j] += (ddir[j] - dir[j] * dd) / len;
}

int orc_project_backward(int n, const float *means, const float *scales, const float *quats,
                         const float *sh, int sh_degree, const orc_camera *cam, const orc_kernel *k,
                         const int *culled, const int *clampxy, const unsigned char *clamped,
                         const double *grad2d, double *dmeans, double *dscales, double *dquats,
                         double *dopac, double *dsh)
{
    const int Kc = (sh_degree + 1) * (sh_degree + 1);
    double cc[3];
    camera_centre(cam, cc);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double *dm = dmeans + 3 * (size_t)i, *ds = dscales + 3 * (size_t)i, *dq = dquats + 4 * (size_t)i;
        double *dshi = dsh + (size_t)Kc * 3 * i;
        if (culled[i]) {
            memset(dm, 0, 3 * sizeof(double));
            memset(ds, 0, 3 * sizeof(double));
            memset(dq, 0, 4 * sizeof(double));
            memset(dshi, 0, (size_t)Kc * 3 * sizeof(double));
            dopac[i] = 0.0;
            continue;
        }
        backward_splat(means + 3 * (size_t)i, scales + 3 * (size_t)i, quats + 4 * (size_t)i,
                       sh + (size_t)Kc * 3 * i, sh_degree, cam, (double)k->psi, clampxy[2 * (size_t)i],
                       clampxy[2 * (size_t)i + 1], clamped[i], cc, grad2d + 9 * (size_t)i, dm, ds, dq, dshi);
        dopac[i] = grad2d[9 * (size_t)i + 5];
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
