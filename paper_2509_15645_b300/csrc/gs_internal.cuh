// gs_internal.cuh -- device-side data structures and the per-Gaussian / per-pixel
// arithmetic shared by the kernels of the 3DGS training hot path (GS-Scale,
// arXiv 2509.15645, §2.4 steps 1-6 and §4.3).  Everything here is FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs_b300.h"

namespace gs {

constexpr int ROW_MEAN = 0, ROW_LS = 3, ROW_QUAT = 6, ROW_OPAC = 10, N_GEO = 11;
constexpr int MAX_VIEWS = 8;
constexpr int LUT_N = 16;       // counter values 0..15 (4-bit counter of §4.3.2)
constexpr int N_GROUPS = 6;     // lr groups: mean, log-scale, quat, opacity, SH DC, SH rest
constexpr int CHUNK = 2048;     // Gaussians per compaction chunk (64 mask words)
constexpr int CHUNK_WORDS = CHUNK / 32;

// Camera as the kernels read it: the API camera plus derived constants.
struct DevCam {
    float R[9], t[3];
    float fx, fy, cx, cy, near_z, far_z;
    float limx, limy;            // guard band: 1.3 * tan(half fov)
    float campos[3];             // camera centre in world space
    int width, height, tile_w, tile_h, tiles_x, tiles_y;
    float loss_inv;              // 1 / (3 W H) of the full image (a region's loss is part of it)
};
// Kernels copy a camera into shared memory one 32-bit word per thread, with
// blocks of at least one warp.
static_assert(sizeof(DevCam) % 4 == 0 && sizeof(DevCam) <= 32 * 4, "DevCam must fit one warp's word copy");

// Restore tables of the deferred update (Fig. 10, §4.3.2) for one step t.
struct DevLut {
    float param[N_GROUPS][LUT_N];   // param_lut[d] (contains lr)
    uint32_t seed;                  // stochastic-rounding seed (BF16 storage)
    int stochastic;                 // 1: BF16 stores round stochastically
    float mom[LUT_N], var[LUT_N];   // b1^(d+1), b2^(d+1)
    float step_size[N_GROUPS];      // lr / (1 - b1^t)
    float bias_corr;                // sqrt(1 - b2^t)
    float inv_bias_corr;            // 1 / sqrt(1 - b2^t)
    float omb1, omb2, eps;          // 1 - b1, 1 - b2, eps
    float b1, b2;
    int max_defer;
    int step;                       // t
    int restore;                    // 0: render/cull without restore
    float decay[N_GROUPS][LUT_N];   // AdamW: (1 - lr wd)^d of the restore; 1 otherwise
    float wdf[N_GROUPS];            // AdamW: 1 - lr wd of the current step; 1 otherwise
};

struct DevArgs {
    DevCam cam[MAX_VIEWS];
    const float *target[MAX_VIEWS];
    DevLut lut;
    int n_views;
};

// Device-resident counters and status (one per context).
struct Counters {
    int n_vis;        // last cull
    int n_keys;       // last render
    int n_upd;        // last deferred Adam update set
    int status;       // first latched gs_status
    float loss;       // last loss
    int n_union;      // gs_step: union of the views' visible sets
    int n_fix;        // last render: Gaussians projected through the FP64 chain
    int n_cand;       // last gs_step cull: Gaussians that passed the visibility pre-test
};

__device__ __forceinline__ void latch(int *status, int code) { atomicCAS(status, 0, code); }

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory by the TMA engine, completing on an
// mbarrier (transaction count = bytes).  Addresses 16-byte aligned, sizes a
// multiple of 16.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the copy engine (async proxy).
__device__ __forceinline__ void fence_barrier_init() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for phase `parity` of a barrier, giving up after `limit` polls
// (returns false then; the caller reports and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t k = 0; k < limit; k++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__host__ __device__ __forceinline__ int lr_group(int row)
{
    return row < 3 ? 0 : row < 6 ? 1 : row < 10 ? 2 : row == 10 ? 3 : row < 14 ? 4 : 5;
}

// ---------------------------------------------------------------------------
// Storage of SH planes and moments: fp32, or bf16 (precision form).  Loads
// widen to fp32; bf16 stores round to nearest or stochastically with a
// counter-based hash of (seed, step, plane, index), so a run is reproducible.
__device__ __forceinline__ float ld_val(const float *p) { return *p; }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// 32-bit integer finaliser (xor-shift / multiply rounds; the "lowbias32"
// constants published by C. Wellons): a counter-based source of the random
// bits of stochastic rounding.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Random bits of the stores of parameter plane `plane` at Gaussian i in one
// step: sr_bits(sr_plane_key(seed, step, plane), i).  The low 16 bits round m,
// the high 16 bits v, and sr_w_bits() of them the weight.
__device__ __forceinline__ uint32_t sr_plane_key(uint32_t seed, uint32_t step, uint32_t plane)
{
    return mix32(plane * 0x85ebca77u ^ mix32(step * 0xc2b2ae3du ^ seed));
}
__device__ __forceinline__ uint32_t sr_bits(uint32_t key, uint32_t i) { return mix32(i * 0x9e3779b1u ^ key); }
__device__ __forceinline__ uint32_t sr_w_bits(uint32_t bits) { return (bits * 0x2c1b3c6du) >> 16; }

// Stores return the value as stored (after rounding).
__device__ __forceinline__ float st_val(float *p, float x, bool, uint32_t)
{
    *p = x;
    return x;
}

// Stochastic rounding: adding 16 random bits below the kept mantissa carries
// into it with probability equal to the dropped fraction (same for both signs,
// the format being sign-magnitude).
__device__ __forceinline__ float st_val(__nv_bfloat16 *p, float x, bool stochastic, uint32_t rnd)
{
    uint32_t u = __float_as_uint(x);
    __nv_bfloat16 b;
    if (!stochastic || (u & 0x7f800000u) == 0x7f800000u) {
        b = __float2bfloat16_rn(x);
    } else {
        u += rnd & 0xffffu;
        b = __ushort_as_bfloat16((unsigned short)(u >> 16));
    }
    *p = b;
    return __bfloat162float(b);
}

// ---------------------------------------------------------------------------
// Deferred restore (Eq. 3 with eps factored out): the current value of a
// parameter whose last d updates were deferred.  d = 0 leaves it untouched.
// The restore direction m / (sqrt(v) + eps) is kept per parameter by the
// optimizer (the scene's rdir planes) so that the restore is one FMA; the two
// helpers below are the only places either quantity is formed, so a stored
// direction and a recomputed one give the same restored value bit for bit.
// Square root by the hardware approximation (PTX sqrt.approx.f32, a few ulps;
// no denormal flush): the optimizer's divisors sqrt(v) + eps need no IEEE
// rounding, and one helper keeps every restore direction the same bit for bit.
__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Optimizer kinds as template arguments (GS_OPT_ADAM, GS_OPT_ADAMW,
// GS_OPT_SGDM): each kernel that restores or steps is compiled per kind, so
// Adam's code has no trace of the others.
// Adam and AdamW restore along m / (sqrt(v) + eps); momentum SGD along its
// buffer b (held in the m planes), exactly.
template <int OPT = GS_OPT_ADAM>
__device__ __forceinline__ float restore_dir(float m, float v, float eps)
{
    if (OPT == GS_OPT_SGDM) return m;
    return __fdividef(m, sqrt_fast(v) + eps);
}

// w <- dec w - plut dir for a delay d > 0 (dec, the decay of the deferred
// steps, only for AdamW).
template <int OPT = GS_OPT_ADAM>
__device__ __forceinline__ float restore_with_dir(float w, float dir, float plut, float dec, int d)
{
    if (OPT == GS_OPT_ADAMW) return d ? __fmaf_rn(-plut, dir, __fmul_rn(dec, w)) : w;
    return d ? __fmaf_rn(-plut, dir, w) : w;
}

template <int OPT = GS_OPT_ADAM>
__device__ __forceinline__ float restore_param(float w, float m, float v, float plut, float dec, int d, float eps)
{
    return d ? restore_with_dir<OPT>(w, restore_dir<OPT>(m, v, eps), plut, dec, d) : w;
}

// ---------------------------------------------------------------------------
// Projection of one Gaussian (§2.4 step 1), FP32.  The cull and the render
// call the same function so that their visibility decisions coincide.
struct Proj {
    float p[3];            // camera-space mean
    float s[3];            // scales
    float qh[4], qn;       // normalised quaternion and the norm
    float Rq[9];           // rotation of the Gaussian
    float T[6];            // J W (2 x 3)
    float S3[6];           // Sigma3: xx, xy, xz, yy, yz, zz
    float a, b, c, det;    // Sigma2 (with low-pass) and its determinant
    float conA, conB, conC;
    float mx, my, radius;
    int cu, cw;            // guard-band clamps
    int rect[4];
    int keep;
    int fp64;              // 2D covariance taken from the FP64 chain
};

__device__ __forceinline__ void quat_rot(const float q[4], float R[9])
{
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// g[0..9] = mean(3), log-scale(3), quaternion(4).
// ---------------------------------------------------------------------------
// FP64 covariance chain for badly conditioned Gaussians (see project_gaussian).
// Used by the fix-up kernels only, so the FP32 kernels keep their register
// budget; both take the FP32 inputs (mean, log-scale, quaternion) and the view.
struct Cov64 {
    double Rq[9], s[3], qh[4], qn, S3[9], T[6], p[3], a, b, c;
    int cu, cw;
};
struct Geo10 {
    float v[10];
};
struct Sym2d {
    double a, b, c;
};
struct CovGrad {
    float gp[3], gls[3], gq[4];
};

static __device__ __forceinline__ void cov_chain_fp64(const Geo10 &G, const DevCam &cam, Cov64 &C)
{
    const float *g = G.v;
    for (int k = 0; k < 3; k++) C.s[k] = exp((double)g[3 + k]);
    double q[4] = {g[6], g[7], g[8], g[9]};
    const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (qq > 0.0) {
        C.qn = sqrt(qq);
        for (int k = 0; k < 4; k++) C.qh[k] = q[k] / C.qn;
    } else {
        C.qn = 1.0; C.qh[0] = 1.0; C.qh[1] = C.qh[2] = C.qh[3] = 0.0;
    }
    const double w = C.qh[0], x = C.qh[1], y = C.qh[2], z = C.qh[3];
    const double Rq[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                          2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                          2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int k = 0; k < 9; k++) C.Rq[k] = Rq[k];
    double M[9];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) M[r * 3 + c] = Rq[r * 3 + c] * C.s[c];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            C.S3[r * 3 + c] = M[r * 3 + 0] * M[c * 3 + 0] + M[r * 3 + 1] * M[c * 3 + 1] + M[r * 3 + 2] * M[c * 3 + 2];
    const float *R = cam.R;
    for (int r = 0; r < 3; r++)
        C.p[r] = (double)R[r * 3 + 0] * g[0] + (double)R[r * 3 + 1] * g[1] + (double)R[r * 3 + 2] * g[2] + (double)cam.t[r];
    const double iz = 1.0 / C.p[2];
    const double u = C.p[0] * iz, v = C.p[1] * iz;
    C.cu = (u < -(double)cam.limx) || (u > (double)cam.limx);
    C.cw = (v < -(double)cam.limy) || (v > (double)cam.limy);
    const double tu = fmin((double)cam.limx, fmax(-(double)cam.limx, u));
    const double tv = fmin((double)cam.limy, fmax(-(double)cam.limy, v));
    const double J00 = cam.fx * iz, J02 = -cam.fx * tu * iz, J11 = cam.fy * iz, J12 = -cam.fy * tv * iz;
    for (int c = 0; c < 3; c++) {
        C.T[c] = J00 * R[c] + J02 * R[6 + c];
        C.T[3 + c] = J11 * R[3 + c] + J12 * R[6 + c];
    }
    double U[6];               // S3 T^T, columns for the two rows of T
    for (int r = 0; r < 3; r++) {
        U[r] = C.S3[r * 3 + 0] * C.T[0] + C.S3[r * 3 + 1] * C.T[1] + C.S3[r * 3 + 2] * C.T[2];
        U[3 + r] = C.S3[r * 3 + 0] * C.T[3] + C.S3[r * 3 + 1] * C.T[4] + C.S3[r * 3 + 2] * C.T[5];
    }
    C.a = C.T[0] * U[0] + C.T[1] * U[1] + C.T[2] * U[2] + 0.3;
    C.b = C.T[0] * U[3] + C.T[1] * U[4] + C.T[2] * U[5];
    C.c = C.T[3] * U[3] + C.T[4] * U[4] + C.T[5] * U[5] + 0.3;
}

static __device__ __forceinline__ Sym2d cov2d_fp64(const Geo10 G, const DevCam &cam)
{
    Cov64 C;
    cov_chain_fp64(G, cam, C);
    return Sym2d{C.a, C.b, C.c};
}

// Adjoint of the chain in FP64: from the gradient of the conic (A, B, C) to
// the camera-space mean (through J only), the log-scales and the quaternion.
static __device__ __forceinline__ CovGrad cov_chain_bwd_fp64(const Geo10 G, const DevCam &cam, float gA, float gB,
                                                          float gC)
{
    CovGrad out;
    float *gp = out.gp, *gls = out.gls, *gq = out.gq;
    Cov64 C;
    cov_chain_fp64(G, cam, C);
    const double a = C.a, b = C.b, c = C.c, det = a * c - b * b, id2 = 1.0 / (det * det);
    const double ga = (-c * c * gA + b * c * gB - b * b * gC) * id2;
    const double gb = (2.0 * b * c * gA - (a * c + b * b) * gB + 2.0 * a * b * gC) * id2;
    const double gc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
    const double hb = 0.5 * gb;
    const double *T = C.T;
    double gS[9];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++)
            gS[r * 3 + q] = ga * T[r] * T[q] + hb * (T[r] * T[3 + q] + T[3 + r] * T[q]) + gc * T[3 + r] * T[3 + q];
    double e0[3], e1[3], gT[6];
    for (int q = 0; q < 3; q++) {
        e0[q] = 2.0 * (ga * T[q] + hb * T[3 + q]);
        e1[q] = 2.0 * (hb * T[q] + gc * T[3 + q]);
    }
    for (int q = 0; q < 3; q++) {
        gT[q] = e0[0] * C.S3[q] + e0[1] * C.S3[3 + q] + e0[2] * C.S3[6 + q];
        gT[3 + q] = e1[0] * C.S3[q] + e1[1] * C.S3[3 + q] + e1[2] * C.S3[6 + q];
    }
    const float *R = cam.R;
    const double gJ00 = gT[0] * R[0] + gT[1] * R[1] + gT[2] * R[2];
    const double gJ02 = gT[0] * R[6] + gT[1] * R[7] + gT[2] * R[8];
    const double gJ11 = gT[3] * R[3] + gT[4] * R[4] + gT[5] * R[5];
    const double gJ12 = gT[3] * R[6] + gT[4] * R[7] + gT[5] * R[8];
    const double iz = 1.0 / C.p[2], iz2 = iz * iz, iz3 = iz2 * iz;
    const double fx = cam.fx, fy = cam.fy;
    double p0 = 0.0, p1 = 0.0, p2 = -(gJ00 * fx + gJ11 * fy) * iz2;
    if (!C.cu) {
        p0 += -gJ02 * fx * iz2;
        p2 += 2.0 * gJ02 * fx * C.p[0] * iz3;
    } else {
        p2 += gJ02 * fx * (C.p[0] > 0.0 ? (double)cam.limx : -(double)cam.limx) * iz2;
    }
    if (!C.cw) {
        p1 += -gJ12 * fy * iz2;
        p2 += 2.0 * gJ12 * fy * C.p[1] * iz3;
    } else {
        p2 += gJ12 * fy * (C.p[1] > 0.0 ? (double)cam.limy : -(double)cam.limy) * iz2;
    }
    gp[0] = (float)p0; gp[1] = (float)p1; gp[2] = (float)p2;
    double M[9], gR[9];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) M[r * 3 + q] = C.Rq[r * 3 + q] * C.s[q];
    for (int q = 0; q < 3; q++) {
        double gsc = 0.0;
        for (int r = 0; r < 3; r++) {
            const double gm = 2.0 * (gS[r * 3 + 0] * M[q] + gS[r * 3 + 1] * M[3 + q] + gS[r * 3 + 2] * M[6 + q]);
            gsc += gm * C.Rq[r * 3 + q];
            gR[r * 3 + q] = gm * C.s[q];
        }
        gls[q] = (float)(gsc * C.s[q]);
    }
    const double qw = C.qh[0], qx = C.qh[1], qy = C.qh[2], qz = C.qh[3];
    const double dw = -2 * qz * gR[1] + 2 * qy * gR[2] + 2 * qz * gR[3] - 2 * qx * gR[5] - 2 * qy * gR[6] + 2 * qx * gR[7];
    const double dx = 2 * qy * gR[1] + 2 * qz * gR[2] + 2 * qy * gR[3] - 4 * qx * gR[4] - 2 * qw * gR[5] +
                      2 * qz * gR[6] + 2 * qw * gR[7] - 4 * qx * gR[8];
    const double dy = -4 * qy * gR[0] + 2 * qx * gR[1] + 2 * qw * gR[2] + 2 * qx * gR[3] + 2 * qz * gR[5] -
                      2 * qw * gR[6] + 2 * qz * gR[7] - 4 * qy * gR[8];
    const double dz = -4 * qz * gR[0] - 2 * qw * gR[1] + 2 * qx * gR[2] + 2 * qw * gR[3] - 4 * qz * gR[4] +
                      2 * qy * gR[5] + 2 * qx * gR[6] + 2 * qy * gR[7];
    const double dq = dw * qw + dx * qx + dy * qy + dz * qz;
    gq[0] = (float)((dw - qw * dq) / C.qn);
    gq[1] = (float)((dx - qx * dq) / C.qn);
    gq[2] = (float)((dy - qy * dq) / C.qn);
    gq[3] = (float)((dz - qz * dq) / C.qn);
    return out;
}

// Cheap conservative pre-test of project_gaussian's keep decision: false only
// when the full projection would reject the Gaussian.  The largest eigenvalue
// of Sigma2 = T Sigma3 T^T + 0.3 I is at most |T|_F^2 max(s)^2 + 0.3, and the
// radius formula adds at most sqrt(0.1) to it, so the pixel radius is at most
// 3 sqrt(|T|_F^2 max(s)^2 + 0.62) + 1; a square of that half-width around the
// projected mean that misses the tiled image (with a pixel of slack for
// rounding) cannot overlap it.  Same depth test, same Jacobian as
// project_gaussian.
// The camera as the conservative pre-test reads it: six 16-byte vectors in
// shared memory instead of ~24 scalar loads per Gaussian.
struct __align__(16) CullCam {
    float R[9], t[3];
    float near_z, far_z, limx, limy;
    float fx, fy, cx, cy;
    float xmax, ymax, pad0, pad1;   // tiles_x * tile_w + 1, tiles_y * tile_h + 1
};

__device__ __forceinline__ void make_cull_cam(const DevCam &c, CullCam &cc)
{
    for (int k = 0; k < 9; k++) cc.R[k] = c.R[k];
    for (int k = 0; k < 3; k++) cc.t[k] = c.t[k];
    cc.near_z = c.near_z; cc.far_z = c.far_z; cc.limx = c.limx; cc.limy = c.limy;
    cc.fx = c.fx; cc.fy = c.fy; cc.cx = c.cx; cc.cy = c.cy;
    cc.xmax = (float)(c.tiles_x * c.tile_w) + 1.f;
    cc.ymax = (float)(c.tiles_y * c.tile_h) + 1.f;
    cc.pad0 = cc.pad1 = 0.f;
}

// Conservative visibility pre-test on the mean and the largest scale (planes
// 0-5 only): false only if the Gaussian's 3-sigma square, under an upper
// bound of its largest screen-space eigenvalue, misses the tile grid.
__device__ __forceinline__ bool maybe_visible(const float g[6], const CullCam &cc)
{
    const float4 *q = reinterpret_cast<const float4 *>(&cc);
    const float4 a = q[0], b = q[1], c = q[2];
    const float px = a.x * g[0] + a.y * g[1] + a.z * g[2] + c.y;
    const float py = a.w * g[0] + b.x * g[1] + b.y * g[2] + c.z;
    const float pz = b.z * g[0] + b.w * g[1] + c.x * g[2] + c.w;
    const float4 d = q[3];
    if (!(pz > d.x && pz < d.y)) return false;
    const float4 e = q[4], f = q[5];
    const float iz = __fdividef(1.f, pz);
    const float u = px * iz, w = py * iz;
    const float tu = fminf(d.z, fmaxf(-d.z, u));
    const float tw = fminf(d.w, fmaxf(-d.w, w));
    // |T|_F^2 = (fx/z)^2 (1 + tu^2) + (fy/z)^2 (1 + tw^2) for T = J W, W a rotation
    const float fxz = e.x * iz, fyz = e.y * iz;
    const float tn = fxz * fxz * (1.f + tu * tu) + fyz * fyz * (1.f + tw * tw);
    const float smax = __expf(fmaxf(g[3], fmaxf(g[4], g[5])));
    const float rb = 3.f * sqrt_fast(1.001f * (tn * smax * smax) + 0.62f) + 2.f;
    const float mx = e.x * u + e.z, my = e.y * w + e.w;
    return mx + rb > -1.f && mx - rb < f.x && my + rb > -1.f && my - rb < f.y;
}

// Conditioning bound above which the 2D covariance is recomputed in FP64.
constexpr float COND_FP64 = 64.f;

// FP64 = false: the FP32 chain only, P.fp64 flags a Gaussian that needs the
// FP64 one (the cull, whose keep decision is set by the large eigenvalue, and
// the first pass of the gather and of the adjoint, which hand flagged
// Gaussians to a fix-up pass); FP64 = true: the fix-up pass itself.
template <bool FP64 = false>
__device__ __forceinline__ void project_gaussian(const float g[10], const DevCam &cam, Proj &P)
{
    P.keep = 0;
    P.fp64 = 0;
    P.rect[0] = P.rect[1] = P.rect[2] = P.rect[3] = 0;
    const float *R = cam.R;
    P.p[0] = R[0] * g[0] + R[1] * g[1] + R[2] * g[2] + cam.t[0];
    P.p[1] = R[3] * g[0] + R[4] * g[1] + R[5] * g[2] + cam.t[1];
    P.p[2] = R[6] * g[0] + R[7] * g[1] + R[8] * g[2] + cam.t[2];
    float pz = P.p[2];
    if (!(pz > cam.near_z && pz < cam.far_z)) return;
    // hardware approximations (a few ulps) for the transcendental steps: every
    // kernel projects through this one function, so their decisions agree
    P.s[0] = __expf(g[3]); P.s[1] = __expf(g[4]); P.s[2] = __expf(g[5]);
    float qn2 = g[6] * g[6] + g[7] * g[7] + g[8] * g[8] + g[9] * g[9];
    if (qn2 > 0.f) {
        const float inv = rsqrtf(qn2);
        P.qn = qn2 * inv;
        P.qh[0] = g[6] * inv; P.qh[1] = g[7] * inv; P.qh[2] = g[8] * inv; P.qh[3] = g[9] * inv;
    } else {
        P.qn = 1.f; P.qh[0] = 1.f; P.qh[1] = P.qh[2] = P.qh[3] = 0.f;
    }
    quat_rot(P.qh, P.Rq);
    // Sigma3 = M M^T, M = Rq diag(s)
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) M[r * 3 + c] = P.Rq[r * 3 + c] * P.s[c];
    P.S3[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    P.S3[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    P.S3[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    P.S3[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    P.S3[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    P.S3[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float iz = __fdividef(1.f, pz);
    float u = P.p[0] * iz, w = P.p[1] * iz;
    float tu = fminf(cam.limx, fmaxf(-cam.limx, u));
    float tw = fminf(cam.limy, fmaxf(-cam.limy, w));
    P.cu = (u < -cam.limx) || (u > cam.limx);
    P.cw = (w < -cam.limy) || (w > cam.limy);
    float J00 = cam.fx * iz, J02 = -cam.fx * tu * iz;
    float J11 = cam.fy * iz, J12 = -cam.fy * tw * iz;
    // T = J W (W = camera rotation R)
    P.T[0] = J00 * R[0] + J02 * R[6];
    P.T[1] = J00 * R[1] + J02 * R[7];
    P.T[2] = J00 * R[2] + J02 * R[8];
    P.T[3] = J11 * R[3] + J12 * R[6];
    P.T[4] = J11 * R[4] + J12 * R[7];
    P.T[5] = J11 * R[5] + J12 * R[8];
    // Sigma2 = T Sigma3 T^T + 0.3 I
    const float *S = P.S3;
    float u0 = S[0] * P.T[0] + S[1] * P.T[1] + S[2] * P.T[2];
    float u1 = S[1] * P.T[0] + S[3] * P.T[1] + S[4] * P.T[2];
    float u2 = S[2] * P.T[0] + S[4] * P.T[1] + S[5] * P.T[2];
    float v0 = S[0] * P.T[3] + S[1] * P.T[4] + S[2] * P.T[5];
    float v1 = S[1] * P.T[3] + S[3] * P.T[4] + S[4] * P.T[5];
    float v2 = S[2] * P.T[3] + S[4] * P.T[4] + S[5] * P.T[5];
    P.a = P.T[0] * u0 + P.T[1] * u1 + P.T[2] * u2 + 0.3f;
    P.b = P.T[0] * v0 + P.T[1] * v1 + P.T[2] * v2;
    P.c = P.T[3] * v0 + P.T[4] * v1 + P.T[5] * v2 + 0.3f;
    P.det = P.a * P.c - P.b * P.b;
    // Rounding in the chain leaves an absolute error of about u * tr(Sigma3) *
    // |T|_F^2 in a, b and c, so the relative error of det (and of the conic)
    // is about u * (a + c) * tr(Sigma3) * |T|_F^2 / det: large for a
    // near-singular Sigma2 and for a needle seen end-on.  Above 64 (a relative
    // error of a few 1e-6) the chain is redone in FP64 from the FP32 inputs.
    const float tr3 = P.S3[0] + P.S3[3] + P.S3[5];
    const float tn = P.T[0] * P.T[0] + P.T[1] * P.T[1] + P.T[2] * P.T[2] + P.T[3] * P.T[3] + P.T[4] * P.T[4] +
                     P.T[5] * P.T[5];
    P.fp64 = !(P.det * COND_FP64 > (P.a + P.c) * tr3 * tn);
    if (FP64 && P.fp64) {
        Geo10 G;
#pragma unroll
        for (int k = 0; k < 10; k++) G.v[k] = g[k];
        const Sym2d S2 = cov2d_fp64(G, cam);
        const double S2d[3] = {S2.a, S2.b, S2.c};
        const double detd = S2d[0] * S2d[2] - S2d[1] * S2d[1];
        P.a = (float)S2d[0];
        P.b = (float)S2d[1];
        P.c = (float)S2d[2];
        P.det = (float)detd;
        if (!(detd > 0.0)) return;
        P.conA = (float)(S2d[2] / detd);
        P.conB = (float)(-S2d[1] / detd);
        P.conC = (float)(S2d[0] / detd);
    } else {
        if (!(P.det > 0.f)) return;
        float idet = __fdividef(1.f, P.det);
        P.conA = P.c * idet; P.conB = -P.b * idet; P.conC = P.a * idet;
    }
    float mid = 0.5f * (P.a + P.c);
    float lam = mid + sqrt_fast(fmaxf(0.1f, mid * mid - P.det));
    P.radius = ceilf(3.f * sqrt_fast(lam));
    P.mx = cam.fx * u + cam.cx;
    P.my = cam.fy * w + cam.cy;
    float itw = 1.f / (float)cam.tile_w, ith = 1.f / (float)cam.tile_h;
    int x0 = (int)floorf((P.mx - P.radius) * itw), x1 = (int)ceilf((P.mx + P.radius) * itw);
    int y0 = (int)floorf((P.my - P.radius) * ith), y1 = (int)ceilf((P.my + P.radius) * ith);
    x0 = min(max(x0, 0), cam.tiles_x); x1 = min(max(x1, 0), cam.tiles_x);
    y0 = min(max(y0, 0), cam.tiles_y); y1 = min(max(y1, 0), cam.tiles_y);
    P.rect[0] = x0; P.rect[1] = x1; P.rect[2] = y0; P.rect[3] = y1;
    P.keep = (P.radius > 0.f) && (x1 > x0) && (y1 > y0);
}

// ---------------------------------------------------------------------------
// Real spherical harmonics to degree 3 (3DGS ordering and signs) of a unit
// direction; nk = (deg+1)^2 values.
struct SHC {
    static constexpr float c0 = 0.28209479177387814f;
    static constexpr float c1 = 0.4886025119029199f;
    static constexpr float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    static constexpr float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    static constexpr float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
};

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16])
{
    Y[0] = SHC::c0;
    if (deg < 1) return;
    Y[1] = -SHC::c1 * y; Y[2] = SHC::c1 * z; Y[3] = -SHC::c1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SHC::c2a * x * y;
    Y[5] = -SHC::c2a * y * z;
    Y[6] = SHC::c2b * (2.f * zz - xx - yy);
    Y[7] = -SHC::c2a * x * z;
    Y[8] = SHC::c2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -SHC::c3a * y * (3.f * xx - yy);
    Y[10] = SHC::c3b * x * y * z;
    Y[11] = -SHC::c3c * y * (4.f * zz - xx - yy);
    Y[12] = SHC::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -SHC::c3c * x * (4.f * zz - xx - yy);
    Y[14] = SHC::c3e * z * (xx - yy);
    Y[15] = -SHC::c3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k Y_k(x,y,z) h_k with respect to (x, y, z) (independent variables).
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float h[16], float g[3])
{
    g[0] = g[1] = g[2] = 0.f;
    if (deg < 1) return;
    g[0] += -SHC::c1 * h[3];
    g[1] += -SHC::c1 * h[1];
    g[2] += SHC::c1 * h[2];
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    g[0] += SHC::c2a * y * h[4] - SHC::c2a * z * h[7] - 2.f * SHC::c2b * x * h[6] + 2.f * SHC::c2c * x * h[8];
    g[1] += SHC::c2a * x * h[4] - SHC::c2a * z * h[5] - 2.f * SHC::c2b * y * h[6] - 2.f * SHC::c2c * y * h[8];
    g[2] += -SHC::c2a * y * h[5] - SHC::c2a * x * h[7] + 4.f * SHC::c2b * z * h[6];
    if (deg < 3) return;
    g[0] += -SHC::c3a * 6.f * x * y * h[9] + SHC::c3b * y * z * h[10] + SHC::c3c * 2.f * x * y * h[11]
            - 6.f * SHC::c3d * x * z * h[12] - SHC::c3c * (4.f * zz - 3.f * xx - yy) * h[13]
            + 2.f * SHC::c3e * x * z * h[14] - SHC::c3a * (3.f * xx - 3.f * yy) * h[15];
    g[1] += -SHC::c3a * (3.f * xx - 3.f * yy) * h[9] + SHC::c3b * x * z * h[10]
            - SHC::c3c * (4.f * zz - xx - 3.f * yy) * h[11] - 6.f * SHC::c3d * y * z * h[12]
            + SHC::c3c * 2.f * x * y * h[13] - 2.f * SHC::c3e * y * z * h[14] + SHC::c3a * 6.f * x * y * h[15];
    g[2] += SHC::c3b * x * y * h[10] - SHC::c3c * 8.f * y * z * h[11]
            + SHC::c3d * (6.f * zz - 3.f * xx - 3.f * yy) * h[12] - SHC::c3c * 8.f * x * z * h[13]
            + SHC::c3e * (xx - yy) * h[14];
}

// ---------------------------------------------------------------------------
// Per-pixel contribution test and alpha (§2.4 step 3).  The forward and both
// passes of the backward call this one function with the same operands, so
// their discrete decisions agree bit for bit.  Returns alpha, or 0 when the
// Gaussian does not contribute; *G = exp(-sigma), *clamped = 0.999 clamp hit.
constexpr float ALPHA_MAX = 0.999f, ALPHA_MIN = 1.f / 255.f, T_STOP = 1e-4f;

__device__ __forceinline__ float splat_alpha(float4 r0, float4 r1, float px, float py, float &dx, float &dy,
                                             float &G, bool &clamped)
{
    // r0 = (mean x, mean y, radius, opacity), r1 = (A, B, C, depth)
    dx = __fsub_rn(r0.x, px);
    dy = __fsub_rn(r0.y, py);
    if (fabsf(dx) > r0.z || fabsf(dy) > r0.z) return 0.f;
    float sig = __fmaf_rn(r1.y, __fmul_rn(dx, dy),
                          __fmul_rn(0.5f, __fmaf_rn(r1.x, __fmul_rn(dx, dx), __fmul_rn(r1.z, __fmul_rn(dy, dy)))));
    if (sig < 0.f) return 0.f;
    G = __expf(-sig);
    float raw = __fmul_rn(r0.w, G);
    clamped = raw > ALPHA_MAX;
    float alpha = fminf(ALPHA_MAX, raw);
    return alpha < ALPHA_MIN ? 0.f : alpha;
}

// The same test and alpha without branches: identical operations, so identical
// results and decisions; the caller masks with the returned value (0 = no
// contribution).  Used where several pixels per thread are evaluated together.
// The caller has already taken the x half of the square test (|dx| <= r, a
// test shared by a thread's pixel column); only the y half is taken here.
__device__ __forceinline__ float splat_alpha_nb(float4 r0, float4 r1, float dx, float py, float &dy, float &G,
                                               bool &clamped)
{
    dy = __fsub_rn(r0.y, py);
    float sig = __fmaf_rn(r1.y, __fmul_rn(dx, dy),
                          __fmul_rn(0.5f, __fmaf_rn(r1.x, __fmul_rn(dx, dx), __fmul_rn(r1.z, __fmul_rn(dy, dy)))));
    G = __expf(-sig);
    float raw = __fmul_rn(r0.w, G);
    clamped = raw > ALPHA_MAX;
    float alpha = fminf(ALPHA_MAX, raw);
    bool ok = (fabsf(dy) <= r0.z) && (sig >= 0.f) && (alpha >= ALPHA_MIN);
    return ok ? alpha : 0.f;
}

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic (sm_100 and later: add/sub/mul/fma .rn.f32x2 on a
// 64-bit register pair): two independent IEEE operations, each rounded as its
// scalar form, in one instruction.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lo2(f2 r)
{
    float a;
    asm("{ .reg .f32 hi; mov.b64 {%0, hi}, %1; }" : "=f"(a) : "l"(r));
    return a;
}
__device__ __forceinline__ float hi2(f2 r)
{
    float b;
    asm("{ .reg .f32 lo; mov.b64 {lo, %0}, %1; }" : "=f"(b) : "l"(r));
    return b;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// ---------------------------------------------------------------------------
// Host-side launch helpers implemented in the .cu files.
struct Scan;   // fwd

void launch_set_args(const DevArgs &a, DevArgs *dst, cudaStream_t s);

}  // namespace gs
