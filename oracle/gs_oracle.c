/*
 * gs_oracle.c -- plain FP64 CPU oracle of the GS-Scale 3DGS training hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link or call this
 * file; only the tests, the smoke check and the CPU baseline of the benchmark
 * use it.  It shares no code, header or constant generator with the CUDA path.
 *
 * What it computes, per view (GS-Scale §2.4, steps 1-6):
 *   project + frustum cull (3D near/far, then 2D image bounds)  -> orc_project
 *   tile keys and their depth order                              -> orc_build_lists
 *   front-to-back alpha compositing                              -> orc_composite
 *   the same image by brute force over all Gaussians             -> orc_composite_brute
 *   L1 loss and its image gradient                               -> orc_loss_l1
 *   the adjoint of the whole render, to every parameter          -> orc_backward
 *   eager Adam (Eq. 1)                                           -> orc_adam_eager
 *   deferred Adam (Eqs. 2-3, pseudocode of Fig. 10, §4.3.2)      -> orc_adam_deferred
 *   catch-up without a new step (tests only)                     -> orc_adam_materialize
 *
 * The paper gives no rasterizer mathematics: it builds on 3DGS / gsplat.  The
 * projection and compositing below are the public 3DGS formulation written out
 * as mathematics; every constant the paper does not fix is a documented reading
 * (0.3 low-pass, 1.3 guard band, 0.1 eigenvalue floor, 3-sigma radius, 0.999
 * alpha clamp, 1/255 alpha floor, 1e-4 transmittance stop, black background,
 * pixel centres at i+0.5, per-pixel square test |p - mu2d| <= r).
 *
 * Everything is double precision; no blocking, fusion or reordering beyond the
 * definitions.  Loops over Gaussians or pixels that are independent carry an
 * OpenMP pragma (used only to time the baseline on many cores); the backward
 * accumulation over pixels runs on one thread.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- layout
 * Parameters are a structure of arrays P[row * pitch + i] (§2.3: mean 3,
 * scale 3, quaternion 4, opacity 1, SH 3*(L+1)^2).  SH row 11 + 3k + c holds
 * coefficient k of colour channel c. */
enum { R_MEAN = 0, R_LSCALE = 3, R_QUAT = 6, R_OPAC = 10, R_SH = 11 };

typedef struct {
    double R[9];      /* world -> camera rotation, row-major (x right, y down, z forward) */
    double t[3];
    double fx, fy, cx, cy;
    double near_z, far_z;
    int32_t width, height;
    int32_t tile_w, tile_h;
} orc_camera;

/* Everything the rasterizer and the backward need about one Gaussian in one view. */
typedef struct {
    int32_t keep;        /* survives the 3D and the 2D cull */
    int32_t rect[4];     /* tile rectangle x0, x1, y0, y1 (half-open) */
    int32_t clampx, clampy;  /* guard-band clamp active in the Jacobian */
    int32_t rgb_clamped[3];
    int32_t pad;
    double depth;        /* camera-space z */
    double mean2d[2];
    double cov2d[3];     /* a, b, c of the 2D covariance (after the 0.3 low-pass) */
    double conic[3];     /* A, B, C = inverse covariance entries */
    double radius;       /* ceil(3 sqrt(lambda_max)) in pixels */
    double opacity;
    double rgb[3];
    double margin;       /* smallest relative distance of a cull decision to its threshold */
    double depth_f32;    /* depth rounded to float32 (used only for the key) */
    double radius_margin;/* relative distance of 3 sqrt(lambda_max) to the integer ceil() rounds across */
} orc_splat;

static const double ALPHA_MAX = 0.999, ALPHA_MIN = 1.0 / 255.0, T_STOP = 1e-4;
static const double LOWPASS = 0.3, GUARD = 1.3, EIG_FLOOR = 0.1;

static int n_params(int deg) { return 11 + 3 * (deg + 1) * (deg + 1); }
static double rel(double a, double b) { double s = fabs(a) > fabs(b) ? fabs(a) : fabs(b); return s > 0 ? fabs(a - b) / s : 0.0; }
static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }

/* ---------------------------------------------------------------- rotations
 * Unit quaternion (w, x, y, z) -> rotation matrix, row-major. */
static void quat_to_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* d R[e] / d q[j] for the formula above, e = 0..8, j = (w, x, y, z). */
static void quat_to_rot_jac(const double q[4], double dR[9][4])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double J[9][4] = {
        {0, 0, -4 * y, -4 * z},
        {-2 * z, 2 * y, 2 * x, -2 * w},
        {2 * y, 2 * z, 2 * w, 2 * x},
        {2 * z, 2 * y, 2 * x, 2 * w},
        {0, -4 * x, 0, -4 * z},
        {-2 * x, -2 * w, 2 * z, 2 * y},
        {-2 * y, 2 * z, -2 * w, 2 * x},
        {2 * x, 2 * w, 2 * z, 2 * y},
        {0, -4 * x, -4 * y, 0},
    };
    memcpy(dR, J, sizeof(J));
}

/* ---------------------------------------------------------------- spherical harmonics
 * Real spherical harmonics up to degree 3 of a unit direction (x, y, z), in the
 * 3DGS ordering and sign convention, with their gradients with respect to
 * (x, y, z) taken as independent variables. */
static void sh_eval(int deg, const double d[3], double Y[16], double dY[16][3])
{
    const double PI = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    double c0 = 0.5 / sqrt(PI);
    double c1 = sqrt(3.0 / (4 * PI));
    double c2a = sqrt(15.0 / (4 * PI)), c2b = sqrt(5.0 / (16 * PI)), c2c = sqrt(15.0 / (16 * PI));
    double c3a = sqrt(35.0 / (32 * PI)), c3b = sqrt(105.0 / (4 * PI)), c3c = sqrt(21.0 / (32 * PI));
    double c3d = sqrt(7.0 / (16 * PI)), c3e = sqrt(105.0 / (16 * PI));
    memset(Y, 0, 16 * sizeof(double));
    memset(dY, 0, 16 * 3 * sizeof(double));
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = -c1 * y;  dY[1][1] = -c1;
    Y[2] = c1 * z;   dY[2][2] = c1;
    Y[3] = -c1 * x;  dY[3][0] = -c1;
    if (deg < 2) return;
    Y[4] = c2a * x * y;                     dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    Y[5] = -c2a * y * z;                    dY[5][1] = -c2a * z; dY[5][2] = -c2a * y;
    Y[6] = c2b * (2 * z * z - x * x - y * y); dY[6][0] = -2 * c2b * x; dY[6][1] = -2 * c2b * y; dY[6][2] = 4 * c2b * z;
    Y[7] = -c2a * x * z;                    dY[7][0] = -c2a * z; dY[7][2] = -c2a * x;
    Y[8] = c2c * (x * x - y * y);           dY[8][0] = 2 * c2c * x; dY[8][1] = -2 * c2c * y;
    if (deg < 3) return;
    Y[9] = -c3a * y * (3 * x * x - y * y);
    dY[9][0] = -c3a * 6 * x * y; dY[9][1] = -c3a * (3 * x * x - 3 * y * y);
    Y[10] = c3b * x * y * z;
    dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    Y[11] = -c3c * y * (4 * z * z - x * x - y * y);
    dY[11][0] = -c3c * (-2 * x * y); dY[11][1] = -c3c * (4 * z * z - x * x - 3 * y * y); dY[11][2] = -c3c * 8 * y * z;
    Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    dY[12][0] = c3d * (-6 * x * z); dY[12][1] = c3d * (-6 * y * z); dY[12][2] = c3d * (6 * z * z - 3 * x * x - 3 * y * y);
    Y[13] = -c3c * x * (4 * z * z - x * x - y * y);
    dY[13][0] = -c3c * (4 * z * z - 3 * x * x - y * y); dY[13][1] = -c3c * (-2 * x * y); dY[13][2] = -c3c * 8 * x * z;
    Y[14] = c3e * z * (x * x - y * y);
    dY[14][0] = c3e * 2 * x * z; dY[14][1] = -c3e * 2 * y * z; dY[14][2] = c3e * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3 * y * y);
    dY[15][0] = -c3a * (3 * x * x - 3 * y * y); dY[15][1] = -c3a * (-6 * x * y);
}

void orc_sh_basis(int deg, const double *dir, double *Y16, double *dY48)
{
    sh_eval(deg, dir, Y16, (double (*)[3])dY48);
}

/* ---------------------------------------------------------------- projection
 * Intermediates of one Gaussian's projection, kept for the chain rule. */
typedef struct {
    double mu[3], s[3], qn, qh[4], Rq[9], M[9], S3[9];
    double p[3], T[6], S2[4];
    double u, w;          /* p_x/p_z, p_y/p_z */
    double tu, tw;        /* the same clamped to the guard band */
    int cu, cw;
    double det;
    double dir[3], vnorm, Y[16], dY[16][3], rgb_raw[3];
    double o;
} proj_state;

static void camera_center(const orc_camera *cam, double c[3])
{
    for (int i = 0; i < 3; i++)
        c[i] = -(cam->R[0 * 3 + i] * cam->t[0] + cam->R[1 * 3 + i] * cam->t[1] + cam->R[2 * 3 + i] * cam->t[2]);
}

/* Step 1 of §2.4 for Gaussian i: 3D cull, EWA projection, 2D cull, SH colour. */
static void project_one(int deg, const double *P, int64_t pitch, int64_t i, const orc_camera *cam,
                        orc_splat *out, proj_state *st)
{
    proj_state S;
    memset(&S, 0, sizeof(S));
    memset(out, 0, sizeof(*out));
    for (int k = 0; k < 3; k++) {
        S.mu[k] = P[(R_MEAN + k) * pitch + i];
        S.s[k] = exp(P[(R_LSCALE + k) * pitch + i]);
    }
    double q[4];
    for (int k = 0; k < 4; k++) q[k] = P[(R_QUAT + k) * pitch + i];
    S.qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (S.qn > 0) for (int k = 0; k < 4; k++) S.qh[k] = q[k] / S.qn;
    else { S.qh[0] = 1; S.qn = 1; }            /* reading: a zero quaternion is the identity */
    quat_to_rot(S.qh, S.Rq);
    /* Sigma3 = R diag(s^2) R^T = M M^T with M = R diag(s) */
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) S.M[r * 3 + c] = S.Rq[r * 3 + c] * S.s[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += S.M[r * 3 + k] * S.M[c * 3 + k];
            S.S3[r * 3 + c] = acc;
        }
    /* camera space */
    for (int r = 0; r < 3; r++)
        S.p[r] = cam->R[r * 3 + 0] * S.mu[0] + cam->R[r * 3 + 1] * S.mu[1] + cam->R[r * 3 + 2] * S.mu[2] + cam->t[r];
    out->depth = S.p[2];
    out->depth_f32 = (double)(float)S.p[2];
    double margin = dmin(rel(S.p[2], cam->near_z), rel(S.p[2], cam->far_z));
    if (!(S.p[2] > cam->near_z && S.p[2] < cam->far_z)) {   /* 3D frustum cull */
        out->margin = margin;
        if (st) *st = S;
        return;
    }
    double fx = cam->fx, fy = cam->fy, pz = S.p[2];
    S.u = S.p[0] / pz; S.w = S.p[1] / pz;
    double limx = GUARD * (0.5 * cam->width / fx), limy = GUARD * (0.5 * cam->height / fy);
    S.tu = dmin(limx, dmax(-limx, S.u)); S.cu = (S.u < -limx || S.u > limx);
    S.tw = dmin(limy, dmax(-limy, S.w)); S.cw = (S.w < -limy || S.w > limy);
    /* J = d(pixel)/d(p), using the clamped ratios in the third column */
    double J[6] = {fx / pz, 0, -fx * S.tu / pz, 0, fy / pz, -fy * S.tw / pz};
    /* T = J W, W the world->camera rotation */
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += J[r * 3 + k] * cam->R[k * 3 + c];
            S.T[r * 3 + c] = acc;
        }
    /* Sigma2 = T Sigma3 T^T + 0.3 I */
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) acc += S.T[r * 3 + k] * S.S3[k * 3 + l] * S.T[c * 3 + l];
            S.S2[r * 2 + c] = acc + (r == c ? LOWPASS : 0.0);
        }
    double a = S.S2[0], b = S.S2[1], c = S.S2[3];
    out->cov2d[0] = a; out->cov2d[1] = b; out->cov2d[2] = c;
    S.det = a * c - b * b;
    margin = dmin(margin, fabs(S.det) / (fabs(a * c) + 1e-300));
    if (!(S.det > 0)) { out->margin = margin; if (st) *st = S; return; }
    out->conic[0] = c / S.det; out->conic[1] = -b / S.det; out->conic[2] = a / S.det;
    double mid = 0.5 * (a + c);
    double lam = mid + sqrt(dmax(EIG_FLOOR, mid * mid - S.det));
    double r3 = 3.0 * sqrt(lam);
    double r = ceil(r3);
    margin = dmin(margin, fabs(r3 - nearbyint(r3)) / r3);
    out->radius_margin = fabs(r3 - nearbyint(r3)) / r3;
    out->radius = r;
    out->mean2d[0] = fx * S.u + cam->cx;
    out->mean2d[1] = fy * S.w + cam->cy;
    int tiles_x = (cam->width + cam->tile_w - 1) / cam->tile_w;
    int tiles_y = (cam->height + cam->tile_h - 1) / cam->tile_h;
    double bx[4] = {(out->mean2d[0] - r) / cam->tile_w, (out->mean2d[0] + r) / cam->tile_w,
                    (out->mean2d[1] - r) / cam->tile_h, (out->mean2d[1] + r) / cam->tile_h};
    double scale_x = dmax(fabs(out->mean2d[0]) + r, 1.0) / cam->tile_w;
    double scale_y = dmax(fabs(out->mean2d[1]) + r, 1.0) / cam->tile_h;
    for (int k = 0; k < 4; k++)
        margin = dmin(margin, fabs(bx[k] - nearbyint(bx[k])) / (k < 2 ? scale_x : scale_y));
    int x0 = (int)floor(bx[0]), x1 = (int)ceil(bx[1]), y0 = (int)floor(bx[2]), y1 = (int)ceil(bx[3]);
    x0 = x0 < 0 ? 0 : (x0 > tiles_x ? tiles_x : x0);
    x1 = x1 < 0 ? 0 : (x1 > tiles_x ? tiles_x : x1);
    y0 = y0 < 0 ? 0 : (y0 > tiles_y ? tiles_y : y0);
    y1 = y1 < 0 ? 0 : (y1 > tiles_y ? tiles_y : y1);
    out->rect[0] = x0; out->rect[1] = x1; out->rect[2] = y0; out->rect[3] = y1;
    out->margin = margin;
    if (r <= 0 || x1 <= x0 || y1 <= y0) { if (st) *st = S; return; }   /* 2D frustum cull */
    out->keep = 1;
    /* colour from SH in the direction camera -> Gaussian (world space) */
    double cc[3];
    camera_center(cam, cc);
    double v[3] = {S.mu[0] - cc[0], S.mu[1] - cc[1], S.mu[2] - cc[2]};
    S.vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; k++) S.dir[k] = v[k] / S.vnorm;
    sh_eval(deg, S.dir, S.Y, S.dY);
    int nk = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0;
        for (int k = 0; k < nk; k++) acc += S.Y[k] * P[(R_SH + 3 * k + ch) * pitch + i];
        S.rgb_raw[ch] = acc + 0.5;
        out->rgb_clamped[ch] = S.rgb_raw[ch] < 0;
        out->rgb[ch] = S.rgb_raw[ch] < 0 ? 0.0 : S.rgb_raw[ch];
    }
    S.o = 1.0 / (1.0 + exp(-P[R_OPAC * pitch + i]));
    out->opacity = S.o;
    out->clampx = S.cu; out->clampy = S.cw;
    if (st) *st = S;
}

void orc_project(int64_t n, int deg, const double *P, int64_t pitch, const orc_camera *cam, orc_splat *out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) project_one(deg, P, pitch, i, cam, &out[i], NULL);
}

/* ---------------------------------------------------------------- keys and order
 * Step 2 of §2.4: one key per (tile in rect that the Gaussian reaches, Gaussian);
 * key = tile id * 2^32 +
 * bits of the float32 depth; ties broken by ascending Gaussian id. */
typedef struct { uint64_t key; int64_t gid; } orc_key;

static uint32_t f32_bits(double d) { float f = (float)d; uint32_t u; memcpy(&u, &f, 4); return u; }

static int key_cmp(const void *pa, const void *pb)
{
    const orc_key *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->gid < b->gid ? -1 : (a->gid > b->gid ? 1 : 0);
}

/* Reading of §2.4 step 2 (which tiles a Gaussian is binned into): the paper
 * and 3DGS bin a Gaussian into every tile of its rectangle; here a (tile,
 * Gaussian) pair is kept only if the Gaussian can reach alpha >= 1/255
 * somewhere in the tile.  "Somewhere" is the rectangle spanned by the
 * centres of the tile's tile_w x tile_h pixels (the whole tile of the grid,
 * also past the image edge of a ragged last tile), intersected with the
 * Gaussian's 3-sigma square widened by `ext` pixels.  Over that rectangle the
 * largest value of o exp(-sigma) is taken exactly: sigma(d) = 1/2 (A dx^2 +
 * C dy^2) + B dx dy with d = mean2d - p is a positive-definite quadratic
 * (the conic of a kept Gaussian), so its minimum over a rectangle is 0 when
 * d = 0 lies inside and otherwise lies on an edge, where sigma is a convex
 * quadratic in one variable minimised at the clamped stationary point.  A
 * dropped pair has no pixel centre with alpha >= 1/255, so no pixel changes.
 * Returns 0 for an empty intersection. */
static double sigma_at(const double *q, double dx, double dy)
{
    return 0.5 * (q[0] * dx * dx + q[2] * dy * dy) + q[1] * dx * dy;
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

double orc_tile_reach(const orc_splat *g, const orc_camera *cam, int tx, int ty, double ext)
{
    const double X0 = tx * cam->tile_w + 0.5, X1 = X0 + cam->tile_w - 1;
    const double Y0 = ty * cam->tile_h + 0.5, Y1 = Y0 + cam->tile_h - 1;
    const double r = g->radius + ext;
    const double x0 = dmax(X0, g->mean2d[0] - r), x1 = dmin(X1, g->mean2d[0] + r);
    const double y0 = dmax(Y0, g->mean2d[1] - r), y1 = dmin(Y1, g->mean2d[1] + r);
    if (x0 > x1 || y0 > y1) return 0.0;
    /* d = mean2d - p ranges over [dx_lo, dx_hi] x [dy_lo, dy_hi] */
    const double dx_lo = g->mean2d[0] - x1, dx_hi = g->mean2d[0] - x0;
    const double dy_lo = g->mean2d[1] - y1, dy_hi = g->mean2d[1] - y0;
    const double *q = g->conic;
    double smin;
    if (dx_lo <= 0 && dx_hi >= 0 && dy_lo <= 0 && dy_hi >= 0) {
        smin = 0.0;
    } else {
        const double dxe[2] = {dx_lo, dx_hi}, dye[2] = {dy_lo, dy_hi};
        smin = INFINITY;
        for (int k = 0; k < 2; k++) {
            /* edge dx = const: d sigma / d dy = C dy + B dx = 0 */
            const double dy = clampd(-q[1] * dxe[k] / q[2], dy_lo, dy_hi);
            smin = dmin(smin, sigma_at(q, dxe[k], dy));
            /* edge dy = const: d sigma / d dx = A dx + B dy = 0 */
            const double dx = clampd(-q[1] * dye[k] / q[0], dx_lo, dx_hi);
            smin = dmin(smin, sigma_at(q, dx, dye[k]));
        }
        smin = dmax(smin, 0.0);
    }
    return g->opacity * exp(-smin);
}

static int pair_kept(const orc_splat *g, const orc_camera *cam, int tx, int ty)
{
    return orc_tile_reach(g, cam, tx, ty, 0.0) >= ALPHA_MIN;
}

/* orc_tile_reach for n pairs (gid[k], tile[k]). */
void orc_tile_reach_many(int64_t n_pairs, const orc_splat *sp, const orc_camera *cam, const int64_t *gid,
                         const int64_t *tile, double ext, double *out)
{
    const int tiles_x = (cam->width + cam->tile_w - 1) / cam->tile_w;
    for (int64_t k = 0; k < n_pairs; k++)
        out[k] = orc_tile_reach(&sp[gid[k]], cam, (int)(tile[k] % tiles_x), (int)(tile[k] / tiles_x), ext);
}

int64_t orc_count_keys(int64_t n, const orc_splat *sp, const orc_camera *cam)
{
    int64_t K = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!sp[i].keep) continue;
        for (int ty = sp[i].rect[2]; ty < sp[i].rect[3]; ty++)
            for (int tx = sp[i].rect[0]; tx < sp[i].rect[1]; tx++) K += pair_kept(&sp[i], cam, tx, ty);
    }
    return K;
}

/* Writes the sorted (tile, gid) sequence and ranges[2*tile] = [begin, end). */
void orc_build_lists(int64_t n, const orc_splat *sp, const orc_camera *cam,
                     int32_t *key_tile, int64_t *key_gid, int64_t *ranges)
{
    int tiles_x = (cam->width + cam->tile_w - 1) / cam->tile_w;
    int tiles_y = (cam->height + cam->tile_h - 1) / cam->tile_h;
    int64_t K = orc_count_keys(n, sp, cam);
    orc_key *keys = malloc((K ? K : 1) * sizeof(orc_key));
    int64_t o = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!sp[i].keep) continue;
        for (int ty = sp[i].rect[2]; ty < sp[i].rect[3]; ty++)
            for (int tx = sp[i].rect[0]; tx < sp[i].rect[1]; tx++) {
                if (!pair_kept(&sp[i], cam, tx, ty)) continue;
                keys[o].key = ((uint64_t)(ty * tiles_x + tx) << 32) | f32_bits(sp[i].depth);
                keys[o].gid = i;
                o++;
            }
    }
    qsort(keys, K, sizeof(orc_key), key_cmp);
    for (int64_t t = 0; t < 2 * (int64_t)tiles_x * tiles_y; t++) ranges[t] = 0;
    for (int64_t k = 0; k < K; k++) {
        key_tile[k] = (int32_t)(keys[k].key >> 32);
        key_gid[k] = keys[k].gid;
        int32_t t = key_tile[k];
        if (k == 0 || key_tile[k - 1] != t) ranges[2 * t] = k;
        if (k == K - 1 || (int32_t)(keys[k + 1].key >> 32) != t) ranges[2 * t + 1] = k + 1;
    }
    free(keys);
}

/* ---------------------------------------------------------------- compositing
 * Step 3 of §2.4.  Gaussian g contributes to pixel p = (i+0.5, j+0.5) when
 *   |p - mu2d| <= r on both axes, sigma = 1/2 (A dx^2 + C dy^2) + B dx dy >= 0
 *   and alpha = min(0.999, o exp(-sigma)) >= 1/255;
 * compositing runs front to back and stops before a Gaussian that would push
 * the transmittance T (1 - alpha) below 1e-4.  C = sum c alpha T + T_final bg. */
typedef struct {
    double alpha, T, G, dx, dy;
    int64_t gid;
    int clamped;
} contrib;

/* Returns the number of contributors written (<= cap) and the final T. */
static int pixel_walk(const orc_splat *sp, const int64_t *list, int64_t len, double px, double py,
                      contrib *out, int cap, double *T_final, double *margin_out, double C[3], uint64_t *hash)
{
    double T = 1.0, margin = 1e300;
    uint64_t hsh = 1469598103934665603ull;   /* FNV-1a over (id, clamp state) of the contributors */
    int nc = 0;
    C[0] = C[1] = C[2] = 0;
    for (int64_t e = 0; e < len; e++) {
        const orc_splat *g = &sp[list[e]];
        double dx = g->mean2d[0] - px, dy = g->mean2d[1] - py;
        double sigma = 0.5 * (g->conic[0] * dx * dx + g->conic[2] * dy * dy) + g->conic[1] * dx * dy;
        double G = exp(-sigma);
        double raw = g->opacity * G;
        double alpha = dmin(ALPHA_MAX, raw);
        /* margins only of decisions that can change this pixel's value: the
         * square test where the Gaussian would contribute, the 1/255 floor and
         * the transmittance stop (the 0.999 clamp is continuous in value) */
        if (alpha >= ALPHA_MIN && sigma >= 0) {
            double scale = dmax(dmax(fabs(g->mean2d[0]), fabs(g->mean2d[1])), g->radius);
            margin = dmin(margin, fabs(g->radius - fabs(dx)) / scale);
            margin = dmin(margin, fabs(g->radius - fabs(dy)) / scale);
        }
        if (fabs(dx) > g->radius || fabs(dy) > g->radius) continue;
        if (sigma < 0) continue;
        margin = dmin(margin, rel(alpha, ALPHA_MIN));
        if (alpha < ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        margin = dmin(margin, rel(Tn, T_STOP));
        if (Tn < T_STOP) break;
        for (int ch = 0; ch < 3; ch++) C[ch] += g->rgb[ch] * alpha * T;
        hsh = (hsh ^ (uint64_t)(2 * list[e] + (raw > ALPHA_MAX))) * 1099511628211ull;
        if (out && nc < cap) {
            out[nc].alpha = alpha; out[nc].T = T; out[nc].G = G;
            out[nc].dx = dx; out[nc].dy = dy; out[nc].gid = list[e];
            out[nc].clamped = raw > ALPHA_MAX;
        }
        nc++;
        T = Tn;
    }
    *T_final = T;
    if (margin_out) *margin_out = margin;
    if (hash) *hash = hsh;
    return nc;
}

/* image[ch*H*W + y*W + x]; bg is the background colour (3). */
void orc_composite(int64_t n, const orc_splat *sp, const orc_camera *cam, const int64_t *key_gid,
                   const int64_t *ranges, const double *bg, double *image, int32_t *n_contrib,
                   double *T_final, double *margin, uint64_t *dhash)
{
    int W = cam->width, H = cam->height;
    int tiles_x = (W + cam->tile_w - 1) / cam->tile_w;
    (void)n;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int t = (y / cam->tile_h) * tiles_x + (x / cam->tile_w);
            int64_t b = ranges[2 * t], e = ranges[2 * t + 1];
            double C[3], T, mg;
            uint64_t hs;
            int nc = pixel_walk(sp, key_gid + b, e - b, x + 0.5, y + 0.5, NULL, 0, &T, &mg, C, &hs);
            if (dhash) dhash[(int64_t)y * W + x] = hs;
            for (int ch = 0; ch < 3; ch++) image[(int64_t)ch * H * W + (int64_t)y * W + x] = C[ch] + T * bg[ch];
            if (n_contrib) n_contrib[(int64_t)y * W + x] = nc;
            if (T_final) T_final[(int64_t)y * W + x] = T;
            if (margin) margin[(int64_t)y * W + x] = mg;
        }
}

/* Brute force: every pixel walks ALL kept Gaussians in (float32 depth, id)
 * order, with no tiles at all. */
static const orc_splat *g_sort_sp;
static int brute_cmp(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    uint32_t ka = f32_bits(g_sort_sp[a].depth), kb = f32_bits(g_sort_sp[b].depth);
    if (ka != kb) return ka < kb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

void orc_composite_brute(int64_t n, const orc_splat *sp, const orc_camera *cam, const double *bg, double *image)
{
    int W = cam->width, H = cam->height;
    int64_t m = 0;
    int64_t *order = malloc((n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) if (sp[i].keep) order[m++] = i;
    g_sort_sp = sp;
    qsort(order, m, sizeof(int64_t), brute_cmp);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double C[3], T;
            pixel_walk(sp, order, m, x + 0.5, y + 0.5, NULL, 0, &T, NULL, C, NULL);
            for (int ch = 0; ch < 3; ch++) image[(int64_t)ch * H * W + (int64_t)y * W + x] = C[ch] + T * bg[ch];
        }
    free(order);
}

/* ---------------------------------------------------------------- loss
 * Step 4 of §2.4 with an L1 loss: L = mean |C - C_gt| over 3HW values;
 * dL/dC = sign(C - C_gt) / (3HW), sign(0) = 0. */
double orc_loss_l1(int64_t count, const double *image, const double *target, double *dimage)
{
    double acc = 0;
    for (int64_t k = 0; k < count; k++) {
        double d = image[k] - target[k];
        acc += fabs(d);
        if (dimage) dimage[k] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)count;
    }
    return acc / (double)count;
}

/* ---------------------------------------------------------------- backward
 * Step 5 of §2.4.  Per pixel with contributors 1..K (in compositing order):
 *   S_i = sum_{j>i} c_j alpha_j T_j + T_{K+1} bg
 *   dL/dc_i     = g alpha_i T_i
 *   dL/dalpha_i = sum_ch g_ch (c_i,ch T_i - S_i,ch / (1 - alpha_i))
 *   alpha = o exp(-sigma) (zero derivative where the 0.999 clamp is active).
 * The per-Gaussian sums then go through the projection by the chain rule. */
static void project_one_backward(int deg, const double *P, int64_t pitch, int64_t i, const orc_camera *cam,
                                 const orc_splat *spl, const proj_state *S, const double g2d[9], double *grad)
{
    /* g2d = dL/d{mean2d x, y, conic A, B, C, opacity, rgb r, g, b} */
    double gmu[3] = {0, 0, 0};
    int nk = (deg + 1) * (deg + 1);
    /* opacity logit: o = sigmoid(l) */
    grad[R_OPAC * pitch + i] += g2d[5] * S->o * (1.0 - S->o);
    /* colour -> SH coefficients and the viewing direction */
    double grgb[3];
    for (int ch = 0; ch < 3; ch++) grgb[ch] = spl->rgb_clamped[ch] ? 0.0 : g2d[6 + ch];
    double gdir[3] = {0, 0, 0};
    for (int k = 0; k < nk; k++)
        for (int ch = 0; ch < 3; ch++) {
            grad[(R_SH + 3 * k + ch) * pitch + i] += S->Y[k] * grgb[ch];
            double coef = P[(R_SH + 3 * k + ch) * pitch + i];
            for (int d = 0; d < 3; d++) gdir[d] += grgb[ch] * coef * S->dY[k][d];
        }
    double dd = gdir[0] * S->dir[0] + gdir[1] * S->dir[1] + gdir[2] * S->dir[2];
    for (int d = 0; d < 3; d++) gmu[d] += (gdir[d] - S->dir[d] * dd) / S->vnorm;
    /* conic (A, B, C) = (c, -b, a) / (ac - b^2) -> covariance (a, b, c) */
    double a = S->S2[0], b = S->S2[1], c = S->S2[3], det = S->det, d2 = det * det;
    double gA = g2d[2], gB = g2d[3], gC = g2d[4];
    double ga = gA * (-c * c / d2) + gB * (b * c / d2) + gC * (-b * b / d2);
    double gb = gA * (2 * b * c / d2) + gB * (-(a * c + b * b) / d2) + gC * (2 * a * b / d2);
    double gc = gA * (-b * b / d2) + gB * (a * b / d2) + gC * (-a * a / d2);
    /* Sigma2 = T Sigma3 T^T + 0.3 I with G2 = dL/dSigma2 (b is one entry shared by both off-diagonals) */
    double G2[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    double gS3[9], gT[6];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) {
            double acc = 0;
            for (int k = 0; k < 2; k++)
                for (int l = 0; l < 2; l++) acc += S->T[k * 3 + r] * G2[k * 2 + l] * S->T[l * 3 + q];
            gS3[r * 3 + q] = acc;
        }
    for (int r = 0; r < 2; r++)
        for (int q = 0; q < 3; q++) {
            double acc = 0;
            for (int k = 0; k < 2; k++)
                for (int l = 0; l < 3; l++) acc += 2.0 * G2[r * 2 + k] * S->T[k * 3 + l] * S->S3[l * 3 + q];
            gT[r * 3 + q] = acc;
        }
    /* T = J W  ->  dL/dJ = dL/dT W^T */
    double gJ[6];
    for (int r = 0; r < 2; r++)
        for (int q = 0; q < 3; q++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += gT[r * 3 + k] * cam->R[q * 3 + k];
            gJ[r * 3 + q] = acc;
        }
    double fx = cam->fx, fy = cam->fy, px = S->p[0], py = S->p[1], pz = S->p[2];
    double gp[3] = {0, 0, 0};
    /* J00 = fx/pz, J11 = fy/pz */
    gp[2] += gJ[0] * (-fx / (pz * pz)) + gJ[4] * (-fy / (pz * pz));
    /* J02 = -fx tu / pz with tu = px/pz unless clamped to a constant */
    if (!S->cu) { gp[0] += gJ[2] * (-fx / (pz * pz)); gp[2] += gJ[2] * (2 * fx * px / (pz * pz * pz)); }
    else        { gp[2] += gJ[2] * (fx * S->tu / (pz * pz)); }
    if (!S->cw) { gp[1] += gJ[5] * (-fy / (pz * pz)); gp[2] += gJ[5] * (2 * fy * py / (pz * pz * pz)); }
    else        { gp[2] += gJ[5] * (fy * S->tw / (pz * pz)); }
    /* mean2d = (fx px/pz + cx, fy py/pz + cy) */
    gp[0] += g2d[0] * fx / pz;
    gp[1] += g2d[1] * fy / pz;
    gp[2] += g2d[0] * (-fx * px / (pz * pz)) + g2d[1] * (-fy * py / (pz * pz));
    /* p = W mu + t */
    for (int d = 0; d < 3; d++)
        gmu[d] += cam->R[0 * 3 + d] * gp[0] + cam->R[1 * 3 + d] * gp[1] + cam->R[2 * 3 + d] * gp[2];
    for (int d = 0; d < 3; d++) grad[(R_MEAN + d) * pitch + i] += gmu[d];
    /* Sigma3 = M M^T -> dL/dM = 2 gS3 M ; M = R diag(s) */
    double gM[9];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += 2.0 * gS3[r * 3 + k] * S->M[k * 3 + q];
            gM[r * 3 + q] = acc;
        }
    double gR[9];
    for (int q = 0; q < 3; q++) {
        double gs = 0;
        for (int r = 0; r < 3; r++) { gs += gM[r * 3 + q] * S->Rq[r * 3 + q]; gR[r * 3 + q] = gM[r * 3 + q] * S->s[q]; }
        grad[(R_LSCALE + q) * pitch + i] += gs * S->s[q];   /* s = exp(log s) */
    }
    double dR[9][4], gqh[4] = {0, 0, 0, 0};
    quat_to_rot_jac(S->qh, dR);
    for (int e = 0; e < 9; e++)
        for (int j = 0; j < 4; j++) gqh[j] += gR[e] * dR[e][j];
    double dq = gqh[0] * S->qh[0] + gqh[1] * S->qh[1] + gqh[2] * S->qh[2] + gqh[3] * S->qh[3];
    for (int j = 0; j < 4; j++) grad[(R_QUAT + j) * pitch + i] += (gqh[j] - S->qh[j] * dq) / S->qn;
    (void)spl;
}

/* grad [D][pitch] is overwritten; splat_grad (optional, [n][9]) receives the
 * per-Gaussian screen-space sums in the order of project_one_backward. */
void orc_backward(int64_t n, int deg, const double *P, int64_t pitch, const orc_camera *cam,
                  const orc_splat *sp, const int64_t *key_gid, const int64_t *ranges, const double *bg,
                  const double *dimage, double *grad, double *splat_grad)
{
    int W = cam->width, H = cam->height, D = n_params(deg);
    int tiles_x = (W + cam->tile_w - 1) / cam->tile_w;
    double *acc = calloc((n ? n : 1) * 9, sizeof(double));
    contrib *cb = NULL;
    int cap = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int t = (y / cam->tile_h) * tiles_x + (x / cam->tile_w);
            int64_t b = ranges[2 * t], e = ranges[2 * t + 1];
            if ((int64_t)cap < e - b) { cap = (int)(e - b); cb = realloc(cb, (cap ? cap : 1) * sizeof(contrib)); }
            double C[3], T;
            int nc = pixel_walk(sp, key_gid + b, e - b, x + 0.5, y + 0.5, cb, cap, &T, NULL, C, NULL);
            double g[3];
            for (int ch = 0; ch < 3; ch++) g[ch] = dimage[(int64_t)ch * H * W + (int64_t)y * W + x];
            /* suffix sums S_i, back to front, in FP64 */
            double Ssum[3] = {T * bg[0], T * bg[1], T * bg[2]};
            for (int k = nc - 1; k >= 0; k--) {
                const contrib *cK = &cb[k];
                const orc_splat *gs = &sp[cK->gid];
                double *A = &acc[cK->gid * 9];
                double dalpha = 0;
                for (int ch = 0; ch < 3; ch++) {
                    A[6 + ch] += g[ch] * cK->alpha * cK->T;
                    dalpha += g[ch] * (gs->rgb[ch] * cK->T - Ssum[ch] / (1.0 - cK->alpha));
                }
                for (int ch = 0; ch < 3; ch++) Ssum[ch] += gs->rgb[ch] * cK->alpha * cK->T;
                if (cK->clamped) continue;              /* alpha = 0.999 does not depend on o or sigma */
                A[5] += dalpha * cK->G;                 /* d alpha / d o = exp(-sigma) */
                double dsig = -cK->alpha * dalpha;      /* d alpha / d sigma = -alpha */
                double dx = cK->dx, dy = cK->dy;
                A[0] += dsig * (gs->conic[0] * dx + gs->conic[1] * dy);
                A[1] += dsig * (gs->conic[1] * dx + gs->conic[2] * dy);
                A[2] += dsig * 0.5 * dx * dx;
                A[3] += dsig * dx * dy;
                A[4] += dsig * 0.5 * dy * dy;
            }
        }
    free(cb);
    for (int r = 0; r < D; r++)
        for (int64_t i = 0; i < n; i++) grad[r * pitch + i] = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!sp[i].keep) continue;
        orc_splat s2;
        proj_state st;
        project_one(deg, P, pitch, i, cam, &s2, &st);
        project_one_backward(deg, P, pitch, i, cam, &sp[i], &st, &acc[i * 9], grad);
    }
    if (splat_grad) memcpy(splat_grad, acc, (size_t)n * 9 * sizeof(double));
    free(acc);
}

/* ---------------------------------------------------------------- Adam
 * Parameter groups for the learning rate: mean, log-scale, quaternion,
 * opacity, SH DC, SH rest. */
static int row_group(int r)
{
    if (r < 3) return 0;
    if (r < 6) return 1;
    if (r < 10) return 2;
    if (r == 10) return 3;
    if (r < 14) return 4;
    return 5;
}

/* Eq. 1 at step t (1-based) for one value. */
static void adam_one(double *w, double *m, double *v, double g, int t, double lr, double b1, double b2, double eps)
{
    *m = b1 * *m + (1 - b1) * g;
    *v = b2 * *v + (1 - b2) * g * g;
    double mhat = *m / (1 - pow(b1, t));
    double vhat = *v / (1 - pow(b2, t));
    *w = *w - lr * mhat / (sqrt(vhat) + eps);
}

/* Eager Adam: every parameter of every Gaussian, gradient g [D][pitch]. */
void orc_adam_eager(int64_t n, int D, int64_t pitch, double *w, double *m, double *v, const double *g,
                    int t, const double *lr, double b1, double b2, double eps)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            adam_one(&w[k], &m[k], &v[k], g[k], t, lr[row_group(r)], b1, b2, eps);
        }
}

/* Lookup tables of the deferred update (Fig. 10, §4.3.2) at step t:
 *   param_lut[0] = 0,
 *   param_lut[i] = (b1/sqrt(b2)) param_lut[i-1]
 *                  + lr b1 / ( sqrt(b2 / (1 - b2^(t-i))) (1 - b1^(t-i)) ),
 *   mom_lut[i] = b1^(i+1), var_lut[i] = b2^(i+1),   i = 0..MAX.
 * Reading: the tables have MAX+1 entries (they are indexed by counter values
 * 0..MAX); entries with i >= t would divide by 1 - b^0 = 0 and can never be
 * used (a delay is at most t-1), so they are left at NaN. */
void orc_adam_lut(int t, double lr, double b1, double b2, int max_defer, double *param_lut, double *mom_lut, double *var_lut)
{
    double scale = b1 / sqrt(b2);
    param_lut[0] = 0;
    for (int i = 1; i <= max_defer; i++) {
        if (i > t - 1) { param_lut[i] = NAN; continue; }
        param_lut[i] = scale * param_lut[i - 1] +
                       (lr * b1) / (sqrt(b2 / (1 - pow(b2, t - i))) * (1 - pow(b1, t - i)));
    }
    for (int i = 0; i <= max_defer; i++) {
        mom_lut[i] = pow(b1, i + 1);
        var_lut[i] = pow(b2, i + 1);
    }
}

/* Deferred Adam at step t.  ids [n_ids] ascending are the Gaussians with a
 * gradient this step (valid_ids), gc [D][n_ids] their gradients.
 *   update_ids = valid_ids U {counter == MAX};
 *   for id in update_ids, with delay d = counter[id]:
 *     mode 0 (tables, Eq. 3 with eps factored out):
 *       m_new = mom_lut[d] m + (1-b1) g ;  v_new = var_lut[d] v + (1-b2) g^2
 *       w    -= param_lut[d] m / (sqrt(v) + eps)            (old m, v)
 *       w     = w - lr/(1-b1^t) m_new / (sqrt(v_new)/sqrt(1-b2^t) + eps)
 *     mode 1 (replay): apply Eq. 1 with g = 0 at steps t-d .. t-1, then Eq. 1
 *       with g at step t -- the exact catch-up.
 *   counter += 1 for every Gaussian, then counter = 0 for update_ids.
 * Reading of the listing: the final division uses sqrt(v_new) (as in Eq. 1),
 * not the stale v.
 * geo_eager != 0: rows 0..9 (mean, scale, quaternion) are updated eagerly for
 * every Gaussian each step (they live on the GPU in §4.2.1); the counter then
 * governs only rows 10.. . */
void orc_adam_deferred(int64_t n, int D, int64_t pitch, double *w, double *m, double *v, uint8_t *counter,
                       const int32_t *ids, int64_t n_ids, const double *gc, int t, const double *lr,
                       double b1, double b2, double eps, int max_defer, int mode, int geo_eager)
{
    double plut[6][16], mlut[16], vlut[16];
    for (int gidx = 0; gidx < 6; gidx++) orc_adam_lut(t, lr[gidx], b1, b2, max_defer, plut[gidx], mlut, vlut);
    double bias_correction = sqrt(1 - pow(b2, t));
    int64_t *slot = malloc((n ? n : 1) * sizeof(int64_t));   /* compact index of i in ids, or -1 */
    for (int64_t i = 0; i < n; i++) slot[i] = -1;
    for (int64_t k = 0; k < n_ids; k++) slot[ids[k]] = k;
    int r0 = geo_eager ? 10 : 0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int in_update = slot[i] >= 0 || counter[i] == max_defer;
        if (geo_eager)
            for (int r = 0; r < 10; r++) {
                double g = slot[i] >= 0 ? gc[r * n_ids + slot[i]] : 0.0;
                int64_t k = r * pitch + i;
                adam_one(&w[k], &m[k], &v[k], g, t, lr[row_group(r)], b1, b2, eps);
            }
        if (!in_update) continue;
        int d = counter[i];
        for (int r = r0; r < D; r++) {
            int64_t k = r * pitch + i;
            double g = slot[i] >= 0 ? gc[r * n_ids + slot[i]] : 0.0;
            double lr_r = lr[row_group(r)];
            if (mode == 1) {
                for (int s = t - d; s < t; s++) adam_one(&w[k], &m[k], &v[k], 0.0, s, lr_r, b1, b2, eps);
                adam_one(&w[k], &m[k], &v[k], g, t, lr_r, b1, b2, eps);
                continue;
            }
            double wk = w[k], mk = m[k], vk = v[k];
            double m_new = mlut[d] * mk + (1 - b1) * g;
            double v_new = vlut[d] * vk + (1 - b2) * g * g;
            m[k] = m_new;
            v[k] = v_new;
            wk -= (plut[row_group(r)][d] * mk) / (sqrt(vk) + eps);
            double step_size = lr_r / (1 - pow(b1, t));
            double denom = sqrt(v_new) / bias_correction + eps;
            w[k] = wk - step_size * m_new / denom;
        }
    }
    for (int64_t i = 0; i < n; i++) {
        int in_update = slot[i] >= 0 || counter[i] == max_defer;
        counter[i] = in_update ? 0 : (uint8_t)(counter[i] + 1);
    }
    free(slot);
}

/* Current (eager-equivalent) state after t_done completed steps, without
 * touching the stored state: m b1^c, v b2^c, w - param_lut_{t_done+1}[c] m / (sqrt(v)+eps)
 * (mode 0) or the replay of c zero-gradient steps (mode 1). */
void orc_adam_materialize(int64_t n, int D, int64_t pitch, const double *w, const double *m, const double *v,
                          const uint8_t *counter, int t_done, const double *lr, double b1, double b2, double eps,
                          int max_defer, int mode, int geo_eager, double *w_out, double *m_out, double *v_out)
{
    double plut[6][16], mlut[16], vlut[16];
    for (int gidx = 0; gidx < 6; gidx++) orc_adam_lut(t_done + 1, lr[gidx], b1, b2, max_defer, plut[gidx], mlut, vlut);
    int r0 = geo_eager ? 10 : 0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c = counter[i];
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            double wk = w[k], mk = m[k], vk = v[k];
            if (r >= r0 && c > 0) {
                if (mode == 1) {
                    for (int s = t_done + 1 - c; s <= t_done; s++)
                        adam_one(&wk, &mk, &vk, 0.0, s, lr[row_group(r)], b1, b2, eps);
                } else {
                    wk = wk - plut[row_group(r)][c] * mk / (sqrt(vk) + eps);
                    mk = mk * pow(b1, c);
                    vk = vk * pow(b2, c);
                }
            }
            w_out[k] = wk; m_out[k] = mk; v_out[k] = vk;
        }
    }
}

/* ---------------------------------------------------------------- AdamW, SGD with momentum
 * §4.3 states that the deferral carries over to other momentum optimizers, naming
 * SGD with momentum and AdamW, without formulas; the catch-ups below are derived
 * the same way as Eqs. 2-3: a Gaussian last updated at step s = t - d - 1 whose
 * gradient was zero for the d steps s+1..t-1.
 *
 * AdamW (decoupled decay lambda, rho = 1 - lr lambda): each zero-gradient step j
 * takes w <- rho w, m <- b1 m, v <- b2 v, w <- w - lr mhat / (sqrt(vhat) + eps).
 * With eps factored out of the k-th skipped step as in Eq. 3,
 *   w_{s+d} = rho^d w_s - wlut[d] m_s / (sqrt(v_s) + eps),
 *   wlut[d] = sum_{k=1..d} rho^(d-k) c_k,  c_k = lr b1^k sqrt((1-b2^j)/b2^k) / (1-b1^j), j = s + k.
 * Written over i = t - j (i = 1..d) this is the recursion
 *   wlut[i] = (b1/sqrt(b2)) wlut[i-1] + rho^(i-1) lr b1 / ( sqrt(b2/(1-b2^(t-i))) (1-b1^(t-i)) ),
 * the Adam table of Fig. 10 with the i-th term weighted by rho^(i-1); decay[i] = rho^i.
 * lambda = 0 gives the Adam tables exactly.
 *
 * SGD with momentum mu (no dampening, no weight decay; buffer b starts at 0):
 * each step b <- mu b + g, w <- w - lr b.  Zero-gradient steps give, exactly,
 *   b_{s+d} = mu^d b_s,  w_{s+d} = w_s - slut[d] b_s,  slut[d] = lr (mu + ... + mu^d),
 * so slut[i] = mu slut[i-1] + lr mu and the update step takes b <- mu^(d+1) b + g. */
static void adamw_one(double *w, double *m, double *v, double g, int t, double lr, double b1, double b2,
                      double eps, double wd)
{
    *w *= 1 - lr * wd;      /* decoupled decay first, then the Adam step */
    adam_one(w, m, v, g, t, lr, b1, b2, eps);
}

static void sgdm_one(double *w, double *b, double g, double lr, double mu)
{
    *b = mu * *b + g;
    *w -= lr * *b;
}

void orc_adamw_lut(int t, double lr, double b1, double b2, double wd, int max_defer, double *wlut, double *decay)
{
    double scale = b1 / sqrt(b2), rho = 1 - lr * wd;
    wlut[0] = 0;
    decay[0] = 1;
    for (int i = 1; i <= max_defer; i++) {
        decay[i] = pow(rho, i);
        if (i > t - 1) { wlut[i] = NAN; continue; }
        wlut[i] = scale * wlut[i - 1] +
                  pow(rho, i - 1) * (lr * b1) / (sqrt(b2 / (1 - pow(b2, t - i))) * (1 - pow(b1, t - i)));
    }
}

void orc_sgdm_lut(double lr, double mu, int max_defer, double *slut, double *mom)
{
    slut[0] = 0;
    mom[0] = mu;
    for (int i = 1; i <= max_defer; i++) {
        slut[i] = mu * slut[i - 1] + lr * mu;
        mom[i] = pow(mu, i + 1);
    }
}

void orc_adamw_eager(int64_t n, int D, int64_t pitch, double *w, double *m, double *v, const double *g, int t,
                     const double *lr, double b1, double b2, double eps, double wd)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            adamw_one(&w[k], &m[k], &v[k], g[k], t, lr[row_group(r)], b1, b2, eps, wd);
        }
}

void orc_sgdm_eager(int64_t n, int D, int64_t pitch, double *w, double *b, const double *g, const double *lr,
                    double mu)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            sgdm_one(&w[k], &b[k], g[k], lr[row_group(r)], mu);
        }
}

/* Deferred AdamW / momentum SGD at step t: update set = ids U {counter == MAX},
 * as orc_adam_deferred.  mode 0: the tables above, then the step with the
 * gradient; mode 1: replay of the d zero-gradient steps, then the step. */
void orc_adamw_deferred(int64_t n, int D, int64_t pitch, double *w, double *m, double *v, uint8_t *counter,
                        const int32_t *ids, int64_t n_ids, const double *gc, int t, const double *lr, double b1,
                        double b2, double eps, double wd, int max_defer, int mode)
{
    double wlut[6][16], dec[6][16];
    for (int gidx = 0; gidx < 6; gidx++) orc_adamw_lut(t, lr[gidx], b1, b2, wd, max_defer, wlut[gidx], dec[gidx]);
    int64_t *slot = malloc((n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) slot[i] = -1;
    for (int64_t k = 0; k < n_ids; k++) slot[ids[k]] = k;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        if (!(slot[i] >= 0 || counter[i] == max_defer)) continue;
        int d = counter[i];
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            int grp = row_group(r);
            double g = slot[i] >= 0 ? gc[r * n_ids + slot[i]] : 0.0;
            if (mode == 1) {
                for (int s = t - d; s < t; s++) adamw_one(&w[k], &m[k], &v[k], 0.0, s, lr[grp], b1, b2, eps, wd);
            } else if (d > 0) {
                w[k] = dec[grp][d] * w[k] - wlut[grp][d] * m[k] / (sqrt(v[k]) + eps);
                m[k] *= pow(b1, d);
                v[k] *= pow(b2, d);
            }
            adamw_one(&w[k], &m[k], &v[k], g, t, lr[grp], b1, b2, eps, wd);
        }
    }
    for (int64_t i = 0; i < n; i++) {
        int in_update = slot[i] >= 0 || counter[i] == max_defer;
        counter[i] = in_update ? 0 : (uint8_t)(counter[i] + 1);
    }
    free(slot);
}

void orc_sgdm_deferred(int64_t n, int D, int64_t pitch, double *w, double *b, uint8_t *counter, const int32_t *ids,
                       int64_t n_ids, const double *gc, const double *lr, double mu, int max_defer, int mode)
{
    double slut[6][16], mom[16];
    for (int gidx = 0; gidx < 6; gidx++) orc_sgdm_lut(lr[gidx], mu, max_defer, slut[gidx], mom);
    int64_t *slot = malloc((n ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) slot[i] = -1;
    for (int64_t k = 0; k < n_ids; k++) slot[ids[k]] = k;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        if (!(slot[i] >= 0 || counter[i] == max_defer)) continue;
        int d = counter[i];
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            int grp = row_group(r);
            double g = slot[i] >= 0 ? gc[r * n_ids + slot[i]] : 0.0;
            if (mode == 1) {
                for (int s = 0; s < d; s++) sgdm_one(&w[k], &b[k], 0.0, lr[grp], mu);
                sgdm_one(&w[k], &b[k], g, lr[grp], mu);
            } else {
                w[k] -= slut[grp][d] * b[k];
                b[k] = mom[d] * b[k] + g;
                w[k] -= lr[grp] * b[k];
            }
        }
    }
    for (int64_t i = 0; i < n; i++) {
        int in_update = slot[i] >= 0 || counter[i] == max_defer;
        counter[i] = in_update ? 0 : (uint8_t)(counter[i] + 1);
    }
    free(slot);
}

/* Current (eager-equivalent) AdamW / SGD state after t_done completed steps,
 * stored state untouched (tables, or replay with mode 1). */
void orc_adamw_materialize(int64_t n, int D, int64_t pitch, const double *w, const double *m, const double *v,
                           const uint8_t *counter, int t_done, const double *lr, double b1, double b2, double eps,
                           double wd, int max_defer, int mode, double *w_out, double *m_out, double *v_out)
{
    double wlut[6][16], dec[6][16];
    for (int gidx = 0; gidx < 6; gidx++)
        orc_adamw_lut(t_done + 1, lr[gidx], b1, b2, wd, max_defer, wlut[gidx], dec[gidx]);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c = counter[i];
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            int grp = row_group(r);
            double wk = w[k], mk = m[k], vk = v[k];
            if (c > 0) {
                if (mode == 1) {
                    for (int s = t_done + 1 - c; s <= t_done; s++) adamw_one(&wk, &mk, &vk, 0.0, s, lr[grp], b1, b2, eps, wd);
                } else {
                    wk = dec[grp][c] * wk - wlut[grp][c] * mk / (sqrt(vk) + eps);
                    mk *= pow(b1, c);
                    vk *= pow(b2, c);
                }
            }
            w_out[k] = wk; m_out[k] = mk; v_out[k] = vk;
        }
    }
}

void orc_sgdm_materialize(int64_t n, int D, int64_t pitch, const double *w, const double *b, const uint8_t *counter,
                          const double *lr, double mu, int max_defer, int mode, double *w_out, double *b_out)
{
    double slut[6][16], mom[16];
    for (int gidx = 0; gidx < 6; gidx++) orc_sgdm_lut(lr[gidx], mu, max_defer, slut[gidx], mom);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c = counter[i];
        for (int r = 0; r < D; r++) {
            int64_t k = r * pitch + i;
            int grp = row_group(r);
            double wk = w[k], bk = b[k];
            if (mode == 1) {
                for (int s = 0; s < c; s++) sgdm_one(&wk, &bk, 0.0, lr[grp], mu);
            } else if (c > 0) {
                wk -= slut[grp][c] * bk;
                bk *= pow(mu, c);
            }
            w_out[k] = wk; b_out[k] = bk;
        }
    }
}

int orc_splat_size(void) { return (int)sizeof(orc_splat); }

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
