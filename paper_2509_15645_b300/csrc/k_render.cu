// k_render.cu -- the differentiable tile rasterizer of §2.4 (steps 1-5) on the
// visible subset chosen by the cull.
//
//   k_gather_project  gather of the visible Gaussians' D planes with the
//                     deferred restore (parameter forwarding of §4.2.2 done in
//                     place), EWA projection, SH colour, opacity -> 48 B splat
//                     record, depth and tile rectangle per Gaussian
//   (k_lists.cu)      each tile's list of the splats that can reach it,
//                     sorted front to back
//   k_raster_fwd      one tile per block or per warp; the tile's splats are
//                     staged through shared memory in batches and composited
//                     front to back
//   k_raster_bwd      one front-to-back pass per tile that recomputes each
//                     pixel's transmittance (nothing stored per pixel) and the
//                     colour behind each splat from the forward's final colour;
//                     warp-shuffle reductions before the atomics into the
//                     per-splat screen-space gradients
//   k_project_bwd     chain rule to mean, log-scale, quaternion, opacity logit
//                     and SH coefficients
#include <algorithm>

#include "gs_kernels.cuh"

namespace gs {

constexpr int PROJ_BLOCK = 128;

struct SLutR {
    float param[N_GROUPS][LUT_N];
    float decay[N_GROUPS][LUT_N];
    float eps;
    int restore;
};

template <int DEG, typename T, int OPT>
__global__ void __launch_bounds__(PROJ_BLOCK) k_gather_project(SceneView sc, const int32_t *__restrict__ ids,
                                                               const int *n_vis_p, int cap,
                                                               const DevArgs *__restrict__ args, int view,
                                                               float *__restrict__ compact, float4 *__restrict__ rec0,
                                                               float4 *__restrict__ rec1, float4 *__restrict__ rec2,
                                                               uint32_t *__restrict__ depth, uint2 *__restrict__ rect,
                                                               int *__restrict__ n_fix, int32_t *__restrict__ fix_idx,
                                                               uint8_t *__restrict__ fix_flag, int *__restrict__ n_big,
                                                               int32_t *__restrict__ big_idx)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    constexpr int D = N_GEO + 3 * NK;
    __shared__ DevCam s_cam;
    __shared__ SLutR L;
    if (threadIdx.x < sizeof(DevCam) / 4)
        ((uint32_t *)&s_cam)[threadIdx.x] = ((const uint32_t *)&args->cam[view])[threadIdx.x];
    for (int t = threadIdx.x; t < N_GROUPS * LUT_N; t += blockDim.x) {
        L.param[t / LUT_N][t % LUT_N] = args->lut.param[t / LUT_N][t % LUT_N];
        L.decay[t / LUT_N][t % LUT_N] = args->lut.decay[t / LUT_N][t % LUT_N];
    }
    if (threadIdx.x == 0) {
        L.eps = args->lut.eps;
        L.restore = args->lut.restore && sc.m && sc.v && sc.counter;
    }
    __syncthreads();
    const int n_vis = min(*n_vis_p, cap);
    const int64_t pitch = sc.pitch;
    const int stride = gridDim.x * blockDim.x;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i_next = k < n_vis ? ids[k] : 0;
    for (; k < n_vis; k += stride) {
        // this thread's next id loaded one item ahead (its planes' loads wait on it)
        const int64_t i = i_next;
        if (k + stride < n_vis) i_next = ids[k + stride];
        if (i < 0 || i >= sc.n) {           // caller-supplied id out of range: an empty splat
            rec0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            rec1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            rec2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            depth[k] = 0u;
            rect[k] = make_uint2(0u, 0u);
            fix_flag[k] = 0;
            for (int r = 0; r < D; r++) compact[r * (int64_t)cap + k] = 0.f;
            continue;
        }
        // gather all D planes (with the restore directions, or m and v) before any arithmetic
        const int64_t sb = sc.sh.base(i);                  // element of Gaussian i in the SH planes
        const int64_t sp = sc.sh.ppitch;
        const T *shw = (const T *)sc.sh.w;
        float w[D];
#pragma unroll
        for (int r = 0; r < D; r++)
            w[r] = r < N_GEO ? __ldg(sc.geo + r * pitch + i) : ld_val(shw + (r - N_GEO) * sp + sb);
        if (L.restore) {
            const int d = sc.counter[i];
            if (d) {
                if (sc.sh.current) {
                    // forwarded SH rows are current: only the geometry planes are restored
                    const T *mp = (const T *)sc.m, *vp = (const T *)sc.v;
#pragma unroll
                    for (int r = 0; r < N_GEO; r++) {
                        const float dir = sc.rdir ? __ldg(sc.rdir + r * pitch + i)
                                                  : restore_dir<OPT>(ld_val(mp + r * pitch + i), ld_val(vp + r * pitch + i), L.eps);
                        w[r] = restore_with_dir<OPT>(w[r], dir, L.param[lr_group(r)][d], L.decay[lr_group(r)][d], d);
                    }
                } else if (sc.rdir) {
                    // geometry directions kept; SH directions from m, v (the optimizer keeps none)
                    const T *msh = (const T *)sc.sh.m, *vsh = (const T *)sc.sh.v;
#pragma unroll
                    for (int r = 0; r < D; r++) {
                        if (r < N_GEO) {
                            w[r] = restore_with_dir<OPT>(w[r], __ldg(sc.rdir + r * pitch + i), L.param[lr_group(r)][d],
                                                         L.decay[lr_group(r)][d], d);
                        } else {
                            const float mm = ld_val(msh + (r - N_GEO) * sp + sb), vv = ld_val(vsh + (r - N_GEO) * sp + sb);
                            w[r] = restore_param<OPT>(w[r], mm, vv, L.param[lr_group(r)][d], L.decay[lr_group(r)][d], d,
                                                      L.eps);
                        }
                    }
                } else {
                    const T *mp = (const T *)sc.m, *vp = (const T *)sc.v;
                    const T *msh = (const T *)sc.sh.m, *vsh = (const T *)sc.sh.v;
#pragma unroll
                    for (int r = 0; r < D; r++) {
                        const float mm = r < N_GEO ? ld_val(mp + r * pitch + i) : ld_val(msh + (r - N_GEO) * sp + sb);
                        const float vv = r < N_GEO ? ld_val(vp + r * pitch + i) : ld_val(vsh + (r - N_GEO) * sp + sb);
                        w[r] = restore_param<OPT>(w[r], mm, vv, L.param[lr_group(r)][d], L.decay[lr_group(r)][d], d,
                                                  L.eps);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < D; r++) compact[r * (int64_t)cap + k] = w[r];
        Proj P;
        project_gaussian(w, s_cam, P);
        fix_flag[k] = (uint8_t)P.fp64;
        if (P.fp64) fix_idx[atomicAdd(n_fix, 1)] = k;      // conic, radius and rect redone in FP64
        float vx = w[0] - s_cam.campos[0], vy = w[1] - s_cam.campos[1], vz = w[2] - s_cam.campos[2];
        float ivn = 1.f / sqrtf(vx * vx + vy * vy + vz * vz);
        float Y[16];
        sh_basis(DEG, vx * ivn, vy * ivn, vz * ivn, Y);
        float rgb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < NK; kk++)
#pragma unroll
            for (int c = 0; c < 3; c++) rgb[c] += Y[kk] * w[N_GEO + 3 * kk + c];
#pragma unroll
        for (int c = 0; c < 3; c++) rgb[c] = fmaxf(rgb[c] + 0.5f, 0.f);
        float o = 1.f / (1.f + expf(-w[ROW_OPAC]));
        const float4 r0v = make_float4(P.mx, P.my, P.radius, o), r1v = make_float4(P.conA, P.conB, P.conC, P.p[2]);
        rec0[k] = r0v;
        rec1[k] = r1v;
        rec2[k] = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
        depth[k] = __float_as_uint(P.p[2]);
        // tiles reached: small rectangles are counted and emitted by
        // k_tiles_count / k_tiles_emit; FP64-flagged splats and large rectangles go to the big
        // list (k_big_counts, k_big_emit).  A splat that is not kept gets an
        // empty rectangle, so that every pass sees the same partition.
        if (!P.keep) P.rect[0] = P.rect[1] = P.rect[2] = P.rect[3] = 0;
        if (P.keep && !P.fp64 && (P.rect[1] - P.rect[0]) * (P.rect[3] - P.rect[2]) > BIG_RECT)
            big_idx[atomicAdd(n_big, 1)] = k;
        rect[k] = make_uint2((uint32_t)P.rect[0] | ((uint32_t)P.rect[1] << 16), (uint32_t)P.rect[2] | ((uint32_t)P.rect[3] << 16));
    }
}

// FP64 fix-up of the Gaussians the gather flagged (badly conditioned 2D
// covariance): conic, radius and tile rectangle from the FP64 chain, before
// their keys are counted (k_big_counts).  Opacity, colour and depth are
// unchanged.
__global__ void __launch_bounds__(PROJ_BLOCK) k_fix_project(const float *__restrict__ compact, int cap,
                                                            const int *__restrict__ n_fix,
                                                            const int32_t *__restrict__ fix_idx,
                                                            const DevArgs *__restrict__ args, int view, float4 *rec0,
                                                            float4 *rec1, uint2 *rect, int *n_big, int32_t *big_idx)
{
    __shared__ DevCam s_cam;
    if (threadIdx.x < sizeof(DevCam) / 4)
        ((uint32_t *)&s_cam)[threadIdx.x] = ((const uint32_t *)&args->cam[view])[threadIdx.x];
    __syncthreads();
    const int nf = min(*n_fix, cap);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
        const int k = fix_idx[j];
        float g[N_GEO];
#pragma unroll
        for (int r = 0; r < N_GEO; r++) g[r] = compact[r * (int64_t)cap + k];
        Proj P;
        P.conA = P.conB = P.conC = 0.f;
        project_gaussian<true>(g, s_cam, P);
        const float o = rec0[k].w;
        rec0[k] = make_float4(P.mx, P.my, P.radius, o);
        rec1[k] = make_float4(P.conA, P.conB, P.conC, P.p[2]);
        if (P.keep) big_idx[atomicAdd(n_big, 1)] = k;        // counted by k_big_counts
        else P.rect[0] = P.rect[1] = P.rect[2] = P.rect[3] = 0;
        rect[k] = make_uint2((uint32_t)P.rect[0] | ((uint32_t)P.rect[1] << 16), (uint32_t)P.rect[2] | ((uint32_t)P.rect[3] << 16));
    }
}


// ---------------------------------------------------------------------------
// Rasterizer blocks: one tile per block.  Each thread owns PPT vertically
// adjacent pixels of one column (block = tile pixels / PPT threads), so the
// per-splat warp reductions of the backward are shared by PPT pixels; the
// per-pixel work is branch-free so the PPT dependency chains interleave.  The
// tile's sorted splats stream through shared memory in batches of BATCH
// records.  (PPT, BATCH) is chosen per context by gs_autotune.
__device__ __forceinline__ float block_sum(float x, float *s_red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = x;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_red[k];
    return t;
}


// Stage the tile's list entries [b, b + cnt) into shared memory (the lists
// hold only splats that can reach the tile: k_tiles_emit / k_big_emit).
// WT: the staging belongs to one warp (warp-tile rasterizers), else to the block.
template <bool COLOR, bool INDEX, bool WT = false>
__device__ __forceinline__ int stage_batch(const uint32_t *__restrict__ svals, const float4 *__restrict__ rec0,
                                           const float4 *__restrict__ rec1, const float4 *__restrict__ rec2,
                                           uint32_t b, int cnt, float4 *s0, float4 *s1, float4 *s2, uint32_t *s_k,
                                           uint32_t kcap_vis)
{
    const int t0 = WT ? (int)(threadIdx.x & 31) : (int)threadIdx.x, nt = WT ? 32 : (int)blockDim.x;
    for (int e = t0; e < cnt; e += nt) {
        const uint32_t k = svals[b + e];
        if (k >= kcap_vis) {            // never for a consistent list; an empty splat rather than a stray read
            s0[e] = make_float4(0.f, 0.f, -1.f, 0.f);
            s1[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (COLOR) s2[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (INDEX) s_k[e] = 0u;
            continue;
        }
        s0[e] = rec0[k];
        s1[e] = rec1[k];
        if (COLOR) s2[e] = rec2[k];
        if (INDEX) s_k[e] = k;
    }
    if (WT) __syncwarp();
    else __syncthreads();
    return cnt;
}

// Next (view, tile) item of a persistent rasterizer block, or false when done.
// WT: each warp takes its own items (warp-tile rasterizers).  View v has
// n_first + tiles items: its tiles of more than FIRST_LIST keys first, then
// all its tiles in order, where one of those is passed over (already taken).
template <bool WT = false>
__device__ __forceinline__ bool next_item(const RasterJob &J, int *s_item, int &view, int &tile)
{
    while (true) {
        int item;
        if (WT) {
            __syncwarp();                              // the previous item's staged records are no longer read
            if ((threadIdx.x & 31) == 0) item = atomicAdd(J.work, 1);
            item = __shfl_sync(0xffffffffu, item, 0);
        } else {
            __syncthreads();                           // the previous item's shared data is no longer read
            if (threadIdx.x == 0) *s_item = atomicAdd(J.work, 1);
            __syncthreads();
            item = *s_item;
        }
        int base = 0, nl = 0, idx = -1;
        for (int v = 0; v < J.n_views; v++) {
            const int tiles = J.tile_ofs[v + 1] - J.tile_ofs[v];
            nl = J.n_first[v] ? min(*J.n_first[v], tiles) : 0;
            if (item < base + nl + tiles) {
                view = v;
                idx = item - base;
                break;
            }
            base += nl + tiles;
        }
        if (idx < 0) return false;
        if (idx < nl) {
            tile = J.first_tiles[view][idx];
            return true;
        }
        tile = idx - nl;
        if (nl == 0) return true;
        const uint2 rg = J.ranges[view][tile];
        if ((int)(rg.y - rg.x) <= FIRST_LIST) return true;
    }
}

// NW > 0: warp tiles -- a tile is exactly 32 threads (tile pixels / PPT = 32)
// and each of the block's NW warps takes its own tiles and staging slot, with
// warp-level synchronisation only (one-warp tiles would otherwise be one-warp
// blocks, of which an SM holds at most 32).  Their register budget is set for
// five blocks per SM (measured faster; the backward kept its own budget, as a
// cap there spills).
template <int PPT, int BATCH, int NW = 0>
__global__ void __launch_bounds__(256, NW ? 5 : 1) k_raster_fwd(const RasterJob J, const DevArgs *__restrict__ args,
                                                    int use_target, float *__restrict__ loss)
{
    constexpr bool WT = NW > 0;
    constexpr int NS = WT ? NW : 1;
    __shared__ float4 s0_[NS][BATCH], s1_[NS][BATCH], s2_[NS][BATCH];
    __shared__ float s_red[8];
    __shared__ int s_item;
    const int slot = WT ? (int)(threadIdx.x >> 5) : 0;
    const int tl = WT ? (int)(threadIdx.x & 31) : (int)threadIdx.x;   // thread within the tile
    float4 *s0 = s0_[slot], *s1 = s1_[slot], *s2 = s2_[slot];
    float loss_part = 0.f;
    int view, tile;
    while (next_item<WT>(J, &s_item, view, tile)) {
    const uint2 *__restrict__ ranges = J.ranges[view];
    const uint32_t *__restrict__ svals = J.svals[view];
    const float4 *__restrict__ rec0 = J.rec0[view], *__restrict__ rec1 = J.rec1[view], *__restrict__ rec2 = J.rec2[view];
    const DevCam &cam = args->cam[J.cam0 + view];
    const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
    const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
    const int x = tx0 + tl % tw;
    const int y0 = ty0 + (tl / tw) * PPT;
    const float px = (float)x + 0.5f;
    // pixel rows covered by this warp (uniform): its first thread's row set plus
    // the further thread rows its 32 lanes span
    const int rows_per_warp = (tw >= 32 ? 1 : 32 / tw) * PPT;
    const float wy0 = (float)(ty0 + (((tl >> 5) << 5) / tw) * PPT) + 0.5f;
    const float wy1 = wy0 + (float)(rows_per_warp - 1);
    const uint2 rg = ranges[tile];
    float T[PPT], C0[PPT], C1[PPT], C2[PPT];
    uint32_t live = 0;   // bit j: pixel j still compositing
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        T[j] = 1.f;
        C0[j] = C1[j] = C2[j] = 0.f;
        if (x < W && y0 + j < H) live |= 1u << j;
    }
    for (uint32_t b = rg.x; b < rg.y; b += BATCH) {
        if (WT) {
            if (!__any_sync(0xffffffffu, live != 0)) break;
            __syncwarp();                            // the previous batch is no longer read
        } else if (__syncthreads_count(live != 0) == 0) {
            break;
        }
        const int nb = stage_batch<true, false, WT>(svals, rec0, rec1, rec2, b, min(BATCH, (int)(rg.y - b)), s0, s1,
                                                    s2, nullptr, J.cap[view]);
        for (int e = 0; e < nb && live; e++) {
            const float4 r0 = s0[e];
            // misses this warp's rows (uniform); a warp tile is the whole tile,
            // which every listed splat's square overlaps
            if (!WT && (r0.y + r0.z < wy0 - 1e-3f || r0.y - r0.z > wy1 + 1e-3f)) continue;
            const float dx = __fsub_rn(r0.x, px);
            if (fabsf(dx) > r0.z) continue;                          // square test on x: shared by the column
            const float4 r1 = s1[e];
#pragma unroll
            for (int j = 0; j < PPT; j++) {
                if (!((live >> j) & 1u)) continue;
                float dy, G;
                bool cl;
                const float a = splat_alpha_nb(r0, r1, dx, (float)(y0 + j) + 0.5f, dy, G, cl);
                if (a == 0.f) continue;
                const float Tn = __fmul_rn(T[j], __fsub_rn(1.f, a));
                if (Tn < T_STOP) {
                    live &= ~(1u << j);
                    continue;
                }
                const float4 c = s2[e];
                const float aT = __fmul_rn(a, T[j]);
                C0[j] = __fmaf_rn(c.x, aT, C0[j]);
                C1[j] = __fmaf_rn(c.y, aT, C1[j]);
                C2[j] = __fmaf_rn(c.z, aT, C2[j]);
                T[j] = Tn;
            }
        }
    }
    const int64_t HW = (int64_t)W * H;
    const float inv = cam.loss_inv;
    float *__restrict__ image = J.image[view], *__restrict__ cfinal = J.cfinal[view], *__restrict__ dimage = J.dimage[view];
    const float *target = use_target ? args->target[J.cam0 + view] : nullptr;
    float part = 0.f;
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        const int y = y0 + j;
        if (x < W && y < H) {
            const int64_t pix = (int64_t)y * W + x;
            image[pix] = C0[j];
            image[HW + pix] = C1[j];
            image[2 * HW + pix] = C2[j];
            if (cfinal) {                    // kept for the backward pass
                cfinal[pix] = C0[j];
                cfinal[HW + pix] = C1[j];
                cfinal[2 * HW + pix] = C2[j];
            }
            if (target) {
                float d0 = C0[j] - target[pix], d1 = C1[j] - target[HW + pix], d2 = C2[j] - target[2 * HW + pix];
                dimage[pix] = (d0 > 0.f ? inv : (d0 < 0.f ? -inv : 0.f));
                dimage[HW + pix] = (d1 > 0.f ? inv : (d1 < 0.f ? -inv : 0.f));
                dimage[2 * HW + pix] = (d2 > 0.f ? inv : (d2 < 0.f ? -inv : 0.f));
                part += (fabsf(d0) + fabsf(d1) + fabsf(d2)) * inv;
            }
        }
    }
    loss_part += part;
    }
    // the loss: one sum per warp (warp tiles) or per block, after the last item
    if (use_target) {
        if (WT) {
#pragma unroll
            for (int o = 16; o; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
            if ((threadIdx.x & 31) == 0 && loss_part != 0.f) atomicAdd(loss, loss_part);
        } else {
            __syncthreads();
            const float t = block_sum(loss_part, s_red);
            if (threadIdx.x == 0 && t != 0.f) atomicAdd(loss, t);
        }
    }
}

// A (warp, splat) with at most this many contributing lanes adds each lane's
// sums with its own atomics instead of reducing over the warp: the reduction
// costs ~45 warp instructions, the direct form ~15 whatever the count, while
// the atomics per address grow with it (measured on the 10M step: 3 lanes
// 528 steps/s, 6: 537, 12: 549, 20: 548, all 32: 493).
constexpr int DIRECT_LANES = 12;

// Sum of v[0..7] over the 32 lanes, transposed: after 4 + 2 + 1 exchanges each
// lane holds one index summed over 8 lanes, two more finish the sum.  Lanes
// with (lane & 3) == 0 end with the total of index (lane >> 2).
__device__ __forceinline__ float warp_transpose_sum8(float v[8], int lane)
{
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float send = b4 ? v[i] : v[i + 4], keep = b4 ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        float send = b3 ? v[i] : v[i + 2], keep = b3 ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        float send = b2 ? v[0] : v[1], keep = b2 ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float r = v[0];
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    return r;
}

// emit_splat for sums that are set only in contributing lanes: the other
// lanes' values are replaced by zeros where the warp sums (no zeroing per entry).
__device__ __forceinline__ void emit_splat_sel(float *__restrict__ g9, uint32_t k, bool contrib, float v[9], int lane)
{
    const uint32_t cmask = __ballot_sync(0xffffffffu, contrib);
    if (cmask == 0u) return;
    float *row = g9 + (int64_t)k * G9_STRIDE;
    if (__popc(cmask) <= DIRECT_LANES) {
        if (contrib) {
            atomicAdd(reinterpret_cast<float4 *>(row), make_float4(v[0], v[1], v[2], v[3]));
            atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(v[4], v[5], v[6], v[7]));
            atomicAdd(row + 8, v[8]);
        }
        return;
    }
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = contrib ? v[j] : 0.f;
    float s8 = contrib ? v[8] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) s8 += __shfl_xor_sync(0xffffffffu, s8, o);
    const float sum = warp_transpose_sum8(x, lane);
    const float q1 = __shfl_down_sync(0xffffffffu, sum, 4);
    const float q2 = __shfl_down_sync(0xffffffffu, sum, 8);
    const float q3 = __shfl_down_sync(0xffffffffu, sum, 12);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<float4 *>(row), make_float4(sum, q1, q2, q3));
        atomicAdd(row + 8, s8);
    } else if (lane == 16) {
        atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(sum, q1, q2, q3));
    }
}

// Backward of the compositing (§2.4 step 5), one front-to-back pass per tile
// that recomputes each pixel's transmittance T_i exactly as the forward did
// (same list, same tests, same operations) together with the colour
// accumulated so far, A_i = sum_{j<=i} c_j a_j T_j.  With the forward's final
// colour F (kept per pixel), the colour behind splat i seen through it is
// T_i R_i = (F - A_i) / (1 - a_i), so
//   dL/da_i = g . (T_i c_i - (F - A_i) / (1 - a_i)),   dL/dc_i = g a_i T_i,
// and nothing is replayed or divided back out of T.  A warp sums its lanes'
// contributions to each splat and issues the atomic adds into g9; the sums
// are taken before the conic and the halves of sigma's square terms are
// applied (once per splat, in the projection backward).
// STATS: also count the (pixel, splat) pairs that pass the square test and the
// pairs that contribute (stats[0], stats[1]).
template <int PPT, int BATCH, bool STATS = false, int NW = 0>
__global__ void __launch_bounds__(256) k_raster_bwd(const RasterJob J, const DevArgs *__restrict__ args,
                                                    unsigned long long *stats = nullptr)
{
    constexpr bool WT = NW > 0;
    constexpr int NS = WT ? NW : 1;
    unsigned long long n_sq = 0, n_on = 0, n_empty = 0;
    __shared__ float4 s0_[NS][BATCH], s1_[NS][BATCH], s2_[NS][BATCH];
    __shared__ uint32_t s_k_[NS][BATCH];
    __shared__ int s_item;
    const int slot = WT ? (int)(threadIdx.x >> 5) : 0;
    const int tl = WT ? (int)(threadIdx.x & 31) : (int)threadIdx.x;   // thread within the tile
    float4 *s0 = s0_[slot], *s1 = s1_[slot], *s2 = s2_[slot];
    uint32_t *s_k = s_k_[slot];
    int view, tile;
    while (next_item<WT>(J, &s_item, view, tile)) {
    const uint2 *__restrict__ ranges = J.ranges[view];
    const uint32_t *__restrict__ svals = J.svals[view];
    const float4 *__restrict__ rec0 = J.rec0[view], *__restrict__ rec1 = J.rec1[view], *__restrict__ rec2 = J.rec2[view];
    const float *__restrict__ cfinal = J.cfinal[view], *__restrict__ dimage = J.dimage[view];
    float *__restrict__ g9 = J.g9[view];
    const DevCam &cam = args->cam[J.cam0 + view];
    const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
    const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
    const int x = tx0 + tl % tw;
    const int y0 = ty0 + (tl / tw) * PPT;
    const float px = (float)x + 0.5f;
    // pixel rows covered by this warp (uniform): its first thread's row set plus
    // the further thread rows its 32 lanes span
    const int rows_per_warp = (tw >= 32 ? 1 : 32 / tw) * PPT;
    const float wy0 = (float)(ty0 + (((tl >> 5) << 5) / tw) * PPT) + 0.5f;
    const float wy1 = wy0 + (float)(rows_per_warp - 1);
    const uint2 rg = ranges[tile];
    const int lane = threadIdx.x & 31;
    const int64_t HW = (int64_t)W * H;
    // per pixel: T, g . F (F the forward's final colour), g . A (A the colour
    // accumulated so far, kept only as its product with g)
    float T[PPT], gF[PPT], gA[PPT], g0[PPT], g1[PPT], g2[PPT];
    uint32_t live = 0;
#pragma unroll
    for (int j = 0; j < PPT; j++) {
        T[j] = 1.f;
        gF[j] = gA[j] = g0[j] = g1[j] = g2[j] = 0.f;
        if (x < W && y0 + j < H) {
            live |= 1u << j;
            const int64_t pix = (int64_t)(y0 + j) * W + x;
            g0[j] = dimage[pix];
            g1[j] = dimage[HW + pix];
            g2[j] = dimage[2 * HW + pix];
            gF[j] = g0[j] * cfinal[pix] + g1[j] * cfinal[HW + pix] + g2[j] * cfinal[2 * HW + pix];
        }
    }
    for (uint32_t b = rg.x; b < rg.y; b += BATCH) {
        if (WT) {
            if (!__any_sync(0xffffffffu, live != 0)) break;
            __syncwarp();                            // the previous batch is no longer read
        } else if (__syncthreads_count(live != 0) == 0) {
            break;
        }
        const int nb = stage_batch<true, true, WT>(svals, rec0, rec1, rec2, b, min(BATCH, (int)(rg.y - b)), s0, s1,
                                                   s2, s_k, J.cap[view]);
        for (int e = 0; e < nb; e++) {
            const float4 r0 = s0[e];
            if (!WT && (r0.y + r0.z < wy0 - 1e-3f || r0.y - r0.z > wy1 + 1e-3f)) continue;   // uniform per warp
            const float dx = __fsub_rn(r0.x, px);
            if constexpr (PPT == 1) {
                // one pixel per thread: the sums are set only where the pixel
                // contributes (no zeroing per entry; emit_splat_sel masks the rest)
                float v[9];
                bool contrib = false;
                const float4 r1 = s1[e];
                if (live && fabsf(dx) <= r0.z) {
                    float dy, G;
                    bool cl;
                    const float a = splat_alpha_nb(r0, r1, dx, (float)y0 + 0.5f, dy, G, cl);
                    if (STATS) n_sq += fabsf(dy) <= r0.z ? 1 : 0;
                    if (a != 0.f) {
                        const float Tn = __fmul_rn(T[0], __fsub_rn(1.f, a));
                        if (Tn < T_STOP) {
                            live = 0u;
                        } else {
                            if (STATS) n_on++;
                            contrib = true;
                            const float4 c = s2[e];
                            const float aT = __fmul_rn(a, T[0]);
                            const float gc = __fmaf_rn(g2[0], c.z, __fmaf_rn(g1[0], c.y, __fmul_rn(g0[0], c.x)));
                            gA[0] = __fmaf_rn(aT, gc, gA[0]);
                            const float dLda =
                                __fmaf_rn(T[0], gc, -__fdividef(__fsub_rn(gF[0], gA[0]), __fsub_rn(1.f, a)));
                            v[6] = __fmul_rn(g0[0], aT);
                            v[7] = __fmul_rn(g1[0], aT);
                            v[8] = __fmul_rn(g2[0], aT);
                            const float ds = cl ? 0.f : __fmul_rn(-a, dLda);    // the 0.999 clamp: no derivative
                            v[5] = ds;
                            const float sdx = __fmul_rn(ds, dx), sdy = __fmul_rn(ds, dy);
                            v[0] = sdx;
                            v[1] = sdy;
                            v[2] = __fmul_rn(sdx, dx);
                            v[3] = __fmul_rn(sdx, dy);
                            v[4] = __fmul_rn(sdy, dy);
                            T[0] = Tn;
                        }
                    }
                }
                if (STATS && WT && __ballot_sync(0xffffffffu, contrib) == 0u && lane == 0) n_empty++;
                emit_splat_sel(g9, s_k[e], contrib, v, lane);
                continue;
            }
            // sums over the warp's pixels: ds dx, ds dy, ds dx^2, ds dx dy, ds dy^2,
            // ds, g_r aT, g_g aT, g_b aT (ds = -a dL/da); the mean, conic and
            // opacity gradients are formed from them once per splat (k_project_bwd)
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (live && fabsf(dx) <= r0.z) {
                const float4 r1 = s1[e];
#pragma unroll
                for (int j = 0; j < PPT; j++) {
                    if (!((live >> j) & 1u)) continue;
                    float dy, G;
                    bool cl;
                    const float a = splat_alpha_nb(r0, r1, dx, (float)(y0 + j) + 0.5f, dy, G, cl);
                    if (STATS) n_sq += fabsf(dy) <= r0.z ? 1 : 0;
                    if (a == 0.f) continue;
                    const float Tn = __fmul_rn(T[j], __fsub_rn(1.f, a));
                    if (Tn < T_STOP) {
                        live &= ~(1u << j);
                        continue;
                    }
                    if (STATS) n_on++;
                    contrib = true;
                    const float4 c = s2[e];
                    const float aT = __fmul_rn(a, T[j]);
                    const float gc = __fmaf_rn(g2[j], c.z, __fmaf_rn(g1[j], c.y, __fmul_rn(g0[j], c.x)));
                    gA[j] = __fmaf_rn(aT, gc, gA[j]);
                    // dL/da = g . (T c - (F - A)/(1 - a)), A through this splat
                    const float dLda = __fmaf_rn(T[j], gc, -__fdividef(__fsub_rn(gF[j], gA[j]), __fsub_rn(1.f, a)));
                    v[6] = __fmaf_rn(g0[j], aT, v[6]);
                    v[7] = __fmaf_rn(g1[j], aT, v[7]);
                    v[8] = __fmaf_rn(g2[j], aT, v[8]);
                    if (!cl) {                                   // the 0.999 clamp has no derivative
                        const float ds = __fmul_rn(-a, dLda);
                        v[5] = __fadd_rn(v[5], ds);
                        const float sdx = __fmul_rn(ds, dx), sdy = __fmul_rn(ds, dy);
                        v[0] = __fadd_rn(v[0], sdx);
                        v[1] = __fadd_rn(v[1], sdy);
                        v[2] = __fmaf_rn(sdx, dx, v[2]);
                        v[3] = __fmaf_rn(sdx, dy, v[3]);
                        v[4] = __fmaf_rn(sdy, dy, v[4]);
                    }
                    T[j] = Tn;
                }
            }
            const uint32_t cmask = __ballot_sync(0xffffffffu, contrib);
            if (cmask != 0u && __popc(cmask) <= DIRECT_LANES) {
                // few contributing lanes: each adds its own sums (no warp reduction)
                if (contrib) {
                    float *row = g9 + (int64_t)s_k[e] * G9_STRIDE;
                    atomicAdd(reinterpret_cast<float4 *>(row), make_float4(v[0], v[1], v[2], v[3]));
                    atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(v[4], v[5], v[6], v[7]));
                    if (v[8] != 0.f) atomicAdd(row + 8, v[8]);
                }
            } else if (cmask != 0u) {
                const uint32_t k = s_k[e];
                float s8 = v[8];
#pragma unroll
                for (int o = 16; o; o >>= 1) s8 += __shfl_xor_sync(0xffffffffu, s8, o);
                // lane 4q holds the sum of index q; lanes 0 and 16 gather 0..3 and 4..7
                const float sum = warp_transpose_sum8(v, lane);
                const float q1 = __shfl_down_sync(0xffffffffu, sum, 4);
                const float q2 = __shfl_down_sync(0xffffffffu, sum, 8);
                const float q3 = __shfl_down_sync(0xffffffffu, sum, 12);
                float *row = g9 + (int64_t)k * G9_STRIDE;
                if (lane == 0) {
                    atomicAdd(reinterpret_cast<float4 *>(row), make_float4(sum, q1, q2, q3));
                    if (s8 != 0.f) atomicAdd(row + 8, s8);
                } else if (lane == 16) {
                    atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(sum, q1, q2, q3));
                }
            }
        }
    }
    }
    if (STATS) {
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            n_sq += __shfl_xor_sync(0xffffffffu, n_sq, o);
            n_on += __shfl_xor_sync(0xffffffffu, n_on, o);
        }
        if (lane == 0) {
            atomicAdd(stats, n_sq);
            atomicAdd(stats + 1, n_on);
            if (n_empty) atomicAdd(stats + 2, n_empty);   // held by lane 0 only
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-tile rasterizers over entry pairs (variant 8): a one-warp tile (32
// pixels, one per lane) walks its list two entries at a time.  The staging
// writes entries 2q and 2q + 1 side by side -- five float4 per pair: (mean x,
// mean y), (radius, opacity), (conic A, B), (conic C, blue), (red, green),
// each as the pair's two values -- so one shared-memory load gives two
// operands of a paired f32x2 instruction, and the per-(pixel, splat) terms of
// both entries (alpha, and in the backward the gradient terms) take one
// instruction each.  The transmittance runs through the two entries in order
// with the scalar kernels' operations, so images are the same bit for bit.
constexpr int PAIR_ROWS = 5;

template <int NP, bool INDEX>
__device__ __forceinline__ int stage_pairs(const uint32_t *__restrict__ svals, const float4 *__restrict__ rec0,
                                           const float4 *__restrict__ rec1, const float4 *__restrict__ rec2,
                                           uint32_t b, int cnt, float *q, uint32_t *s_k, uint32_t kcap_vis)
{
    const int lane = threadIdx.x & 31;
    const int padded = (cnt + 1) & ~1;
    for (int e = lane; e < padded; e += 32) {
        float4 r0 = make_float4(0.f, 0.f, -1.f, 0.f), r1 = make_float4(0.f, 0.f, 0.f, 0.f), r2 = r1;
        uint32_t k = 0u;
        if (e < cnt) {
            k = svals[b + e];
            if (k < kcap_vis) {            // else an empty splat (never for a consistent list)
                r0 = rec0[k];
                r1 = rec1[k];
                r2 = rec2[k];
            } else {
                k = 0u;
            }
        }
        const int p = e >> 1, h = e & 1;
        float *q0 = q + (0 * NP + p) * 4, *q1 = q + (1 * NP + p) * 4, *q2 = q + (2 * NP + p) * 4;
        float *q3 = q + (3 * NP + p) * 4, *q4 = q + (4 * NP + p) * 4;
        q0[h] = r0.x; q0[2 + h] = r0.y;
        q1[h] = r0.z; q1[2 + h] = r0.w;
        q2[h] = r1.x; q2[2 + h] = r1.y;
        q3[h] = r1.z; q3[2 + h] = r2.z;
        q4[h] = r2.x; q4[2 + h] = r2.y;
        if (INDEX) s_k[e] = k;
    }
    __syncwarp();
    return padded >> 1;
}

// Alphas of the pair's two entries at pixel (px, py), as splat_alpha_nb
// computes each (same operations, paired).  in0 / in1: the entry passed the
// warp's row test and the pixel's x test.
struct PairAlpha {
    f2 dx2, dy2;
    float a0, a1, G0, G1;
    bool cl0, cl1;
};
__device__ __forceinline__ PairAlpha pair_alpha(const float4 &m, const float4 &ro, const float4 &ab, const float4 &cc,
                                                f2 px2, f2 py2, bool in0, bool in1)
{
    PairAlpha P;
    P.dx2 = sub2(pk2(m.x, m.y), px2);
    P.dy2 = sub2(pk2(m.z, m.w), py2);
    const f2 sig2 = fma2(pk2(ab.z, ab.w), mul2(P.dx2, P.dy2),
                         mul2(pk2(0.5f, 0.5f), fma2(pk2(ab.x, ab.y), mul2(P.dx2, P.dx2),
                                                    mul2(pk2(cc.x, cc.y), mul2(P.dy2, P.dy2)))));
    const float s0 = lo2(sig2), s1 = hi2(sig2);
    P.G0 = __expf(-s0);
    P.G1 = __expf(-s1);
    const f2 raw2 = mul2(pk2(ro.z, ro.w), pk2(P.G0, P.G1));
    const float raw0 = lo2(raw2), raw1 = hi2(raw2);
    P.cl0 = raw0 > ALPHA_MAX;
    P.cl1 = raw1 > ALPHA_MAX;
    const float al0 = fminf(ALPHA_MAX, raw0), al1 = fminf(ALPHA_MAX, raw1);
    const bool ok0 = in0 && fabsf(lo2(P.dy2)) <= ro.x && s0 >= 0.f && al0 >= ALPHA_MIN;
    const bool ok1 = in1 && fabsf(hi2(P.dy2)) <= ro.y && s1 >= 0.f && al1 >= ALPHA_MIN;
    P.a0 = ok0 ? al0 : 0.f;
    P.a1 = ok1 ? al1 : 0.f;
    return P;
}

template <int BATCH, int NW>
__global__ void __launch_bounds__(32 * NW, 4) k_raster_fwd_pairs(const RasterJob J, const DevArgs *__restrict__ args,
                                                                 int use_target, float *__restrict__ loss)
{
    static_assert(BATCH % 2 == 0, "entry pairs");
    constexpr int NP = BATCH / 2;
    __shared__ __align__(16) float q_[NW][PAIR_ROWS * NP * 4];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31;
    float *q = q_[threadIdx.x >> 5];
    const float4 *Q = reinterpret_cast<const float4 *>(q);
    float loss_part = 0.f;
    int view, tile;
    while (next_item<true>(J, &s_item, view, tile)) {
        const uint2 *__restrict__ ranges = J.ranges[view];
        float *__restrict__ image = J.image[view], *__restrict__ cfinal = J.cfinal[view];
        float *__restrict__ dimage = J.dimage[view];
        const DevCam &cam = args->cam[J.cam0 + view];
        const float *target = use_target ? args->target[J.cam0 + view] : nullptr;
        const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
        const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
        const int x = tx0 + lane % tw, y = ty0 + lane / tw;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const float wy0 = (float)ty0 + 0.5f, wy1 = wy0 + (float)(th - 1);
        const f2 px2 = pk2(px, px), py2 = pk2(py, py);
        const uint2 rg = ranges[tile];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        bool live = x < W && y < H;
        for (uint32_t b = rg.x; b < rg.y; b += BATCH) {
            if (!__any_sync(0xffffffffu, live)) break;
            __syncwarp();                            // the previous batch is no longer read
            const int np = stage_pairs<NP, false>(J.svals[view], J.rec0[view], J.rec1[view], J.rec2[view], b,
                                                  min(BATCH, (int)(rg.y - b)), q, nullptr, J.cap[view]);
            for (int p = 0; p < np && live; p++) {
                const float4 m = Q[0 * NP + p], ro = Q[1 * NP + p];
                const bool r0 = !(m.z + ro.x < wy0 - 1e-3f || m.z - ro.x > wy1 + 1e-3f);   // uniform per warp
                const bool r1 = !(m.w + ro.y < wy0 - 1e-3f || m.w - ro.y > wy1 + 1e-3f);
                if (!r0 && !r1) continue;
                const float dx0 = __fsub_rn(m.x, px), dx1 = __fsub_rn(m.y, px);
                const bool in0 = r0 && fabsf(dx0) <= ro.x, in1 = r1 && fabsf(dx1) <= ro.y;
                if (!in0 && !in1) continue;
                const PairAlpha A = pair_alpha(m, ro, Q[2 * NP + p], Q[3 * NP + p], px2, py2, in0, in1);
                if (A.a0 != 0.f) {
                    const float Tn = __fmul_rn(T, __fsub_rn(1.f, A.a0));
                    if (Tn < T_STOP) {
                        live = false;
                        continue;
                    }
                    const float4 c = Q[4 * NP + p], cz = Q[3 * NP + p];
                    const float aT = __fmul_rn(A.a0, T);
                    C0 = __fmaf_rn(c.x, aT, C0);
                    C1 = __fmaf_rn(c.z, aT, C1);
                    C2 = __fmaf_rn(cz.z, aT, C2);
                    T = Tn;
                }
                if (A.a1 != 0.f) {
                    const float Tn = __fmul_rn(T, __fsub_rn(1.f, A.a1));
                    if (Tn < T_STOP) {
                        live = false;
                        continue;
                    }
                    const float4 c = Q[4 * NP + p], cz = Q[3 * NP + p];
                    const float aT = __fmul_rn(A.a1, T);
                    C0 = __fmaf_rn(c.y, aT, C0);
                    C1 = __fmaf_rn(c.w, aT, C1);
                    C2 = __fmaf_rn(cz.w, aT, C2);
                    T = Tn;
                }
            }
        }
        if (x < W && y < H) {
            const int64_t HW = (int64_t)W * H, pix = (int64_t)y * W + x;
            image[pix] = C0;
            image[HW + pix] = C1;
            image[2 * HW + pix] = C2;
            if (cfinal) {
                cfinal[pix] = C0;
                cfinal[HW + pix] = C1;
                cfinal[2 * HW + pix] = C2;
            }
            if (target) {
                const float inv = cam.loss_inv;
                float d0 = C0 - target[pix], d1 = C1 - target[HW + pix], d2 = C2 - target[2 * HW + pix];
                dimage[pix] = (d0 > 0.f ? inv : (d0 < 0.f ? -inv : 0.f));
                dimage[HW + pix] = (d1 > 0.f ? inv : (d1 < 0.f ? -inv : 0.f));
                dimage[2 * HW + pix] = (d2 > 0.f ? inv : (d2 < 0.f ? -inv : 0.f));
                loss_part += (fabsf(d0) + fabsf(d1) + fabsf(d2)) * inv;
            }
        }
    }
    if (use_target) {
#pragma unroll
        for (int o = 16; o; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
        if (lane == 0 && loss_part != 0.f) atomicAdd(loss, loss_part);
    }
}

// A warp's sums for one splat (v as in k_raster_bwd) into its g9 record:
// per-lane atomics when few lanes contribute, else a warp reduction.
__device__ __forceinline__ void emit_splat(float *__restrict__ g9, uint32_t k, bool contrib, float v[9], int lane)
{
    const uint32_t cmask = __ballot_sync(0xffffffffu, contrib);
    if (cmask == 0u) return;
    float *row = g9 + (int64_t)k * G9_STRIDE;
    if (__popc(cmask) <= DIRECT_LANES) {
        if (contrib) {
            atomicAdd(reinterpret_cast<float4 *>(row), make_float4(v[0], v[1], v[2], v[3]));
            atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(v[4], v[5], v[6], v[7]));
            if (v[8] != 0.f) atomicAdd(row + 8, v[8]);
        }
        return;
    }
    float s8 = v[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) s8 += __shfl_xor_sync(0xffffffffu, s8, o);
    const float sum = warp_transpose_sum8(v, lane);
    const float q1 = __shfl_down_sync(0xffffffffu, sum, 4);
    const float q2 = __shfl_down_sync(0xffffffffu, sum, 8);
    const float q3 = __shfl_down_sync(0xffffffffu, sum, 12);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<float4 *>(row), make_float4(sum, q1, q2, q3));
        if (s8 != 0.f) atomicAdd(row + 8, s8);
    } else if (lane == 16) {
        atomicAdd(reinterpret_cast<float4 *>(row + 4), make_float4(sum, q1, q2, q3));
    }
}

template <int BATCH, int NW, bool STATS = false>
__global__ void __launch_bounds__(32 * NW, 4) k_raster_bwd_pairs(const RasterJob J, const DevArgs *__restrict__ args,
                                                             unsigned long long *stats = nullptr)
{
    static_assert(BATCH % 2 == 0, "entry pairs");
    constexpr int NP = BATCH / 2;
    __shared__ __align__(16) float q_[NW][PAIR_ROWS * NP * 4];
    __shared__ uint32_t k_[NW][BATCH];
    __shared__ int s_item;
    unsigned long long n_sq = 0, n_on = 0;
    const int lane = threadIdx.x & 31;
    float *q = q_[threadIdx.x >> 5];
    uint32_t *s_k = k_[threadIdx.x >> 5];
    const float4 *Q = reinterpret_cast<const float4 *>(q);
    int view, tile;
    while (next_item<true>(J, &s_item, view, tile)) {
        const uint2 *__restrict__ ranges = J.ranges[view];
        const float *__restrict__ cfinal = J.cfinal[view], *__restrict__ dimage = J.dimage[view];
        float *__restrict__ g9 = J.g9[view];
        const DevCam &cam = args->cam[J.cam0 + view];
        const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
        const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
        const int x = tx0 + lane % tw, y = ty0 + lane / tw;
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const float wy0 = (float)ty0 + 0.5f, wy1 = wy0 + (float)(th - 1);
        const f2 px2 = pk2(px, px), py2 = pk2(py, py);
        const uint2 rg = ranges[tile];
        float T = 1.f, gF = 0.f, gA = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        bool live = x < W && y < H;
        if (live) {
            const int64_t HW = (int64_t)W * H, pix = (int64_t)y * W + x;
            g0 = dimage[pix];
            g1 = dimage[HW + pix];
            g2 = dimage[2 * HW + pix];
            gF = g0 * cfinal[pix] + g1 * cfinal[HW + pix] + g2 * cfinal[2 * HW + pix];
        }
        const f2 g0_2 = pk2(g0, g0), g1_2 = pk2(g1, g1), g2_2 = pk2(g2, g2);
        for (uint32_t b = rg.x; b < rg.y; b += BATCH) {
            if (!__any_sync(0xffffffffu, live)) break;
            __syncwarp();
            const int np = stage_pairs<NP, true>(J.svals[view], J.rec0[view], J.rec1[view], J.rec2[view], b,
                                                 min(BATCH, (int)(rg.y - b)), q, s_k, J.cap[view]);
            for (int p = 0; p < np; p++) {
                const float4 m = Q[0 * NP + p], ro = Q[1 * NP + p];
                const bool r0 = !(m.z + ro.x < wy0 - 1e-3f || m.z - ro.x > wy1 + 1e-3f);   // uniform per warp
                const bool r1 = !(m.w + ro.y < wy0 - 1e-3f || m.w - ro.y > wy1 + 1e-3f);
                if (!r0 && !r1) continue;
                const float dx0 = __fsub_rn(m.x, px), dx1 = __fsub_rn(m.y, px);
                const bool in0 = live && r0 && fabsf(dx0) <= ro.x;
                bool c0 = false, c1 = false;
                float v0[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float v1[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                const float4 ab = Q[2 * NP + p], cc = Q[3 * NP + p];
                if (in0 || (live && r1 && fabsf(dx1) <= ro.y)) {
                    const bool in1 = live && r1 && fabsf(dx1) <= ro.y;
                    const PairAlpha A = pair_alpha(m, ro, ab, cc, px2, py2, in0, in1);
                    // entry 2p then 2p + 1 through the transmittance, as the scalar kernel
                    if (STATS) n_sq += (in0 && fabsf(lo2(A.dy2)) <= ro.x) ? 1 : 0;
                    float a0 = A.a0, a1 = A.a1;
                    const float T0 = T;
                    if (a0 != 0.f) {
                        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a0));
                        if (Tn < T_STOP) {
                            live = false;
                            a0 = a1 = 0.f;
                        } else {
                            c0 = true;
                            T = Tn;
                        }
                    }
                    if (STATS && live) n_sq += (in1 && fabsf(hi2(A.dy2)) <= ro.y) ? 1 : 0;
                    const float T1 = T;
                    if (live && a1 != 0.f) {
                        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a1));
                        if (Tn < T_STOP) {
                            live = false;
                            a1 = 0.f;
                        } else {
                            c1 = true;
                            T = Tn;
                        }
                    } else {
                        a1 = 0.f;
                    }
                    if (STATS) n_on += (c0 ? 1 : 0) + (c1 ? 1 : 0);
                    if (c0 || c1) {
                        const float4 rg4 = Q[4 * NP + p];
                        const f2 T2 = pk2(T0, T1), a2 = pk2(a0, a1);
                        const f2 aT2 = mul2(a2, T2);
                        const f2 gc2 = fma2(g2_2, pk2(cc.z, cc.w), fma2(g1_2, pk2(rg4.z, rg4.w), mul2(g0_2, pk2(rg4.x, rg4.y))));
                        const float gA0 = __fmaf_rn(lo2(aT2), lo2(gc2), gA);
                        const float gA1 = __fmaf_rn(hi2(aT2), hi2(gc2), gA0);
                        gA = gA1;
                        // dL/da = g . (T c - (F - A)/(1 - a)), A through this splat
                        const float q0 = __fdividef(__fsub_rn(gF, gA0), __fsub_rn(1.f, a0));
                        const float q1 = __fdividef(__fsub_rn(gF, gA1), __fsub_rn(1.f, a1));
                        const f2 dl2 = fma2(T2, gc2, pk2(-q0, -q1));
                        // the 0.999 clamp has no derivative; entries that do not contribute add nothing
                        const f2 dlm2 = pk2(c0 && !A.cl0 ? lo2(dl2) : 0.f, c1 && !A.cl1 ? hi2(dl2) : 0.f);
                        const f2 ds2 = mul2(pk2(-a0, -a1), dlm2);
                        const f2 sdx2 = mul2(ds2, A.dx2), sdy2 = mul2(ds2, A.dy2);
                        const f2 v2 = mul2(sdx2, A.dx2), v3 = mul2(sdx2, A.dy2), v4 = mul2(sdy2, A.dy2);
                        const f2 v6 = mul2(g0_2, aT2), v7 = mul2(g1_2, aT2), v8 = mul2(g2_2, aT2);
                        v0[0] = lo2(sdx2); v1[0] = hi2(sdx2);
                        v0[1] = lo2(sdy2); v1[1] = hi2(sdy2);
                        v0[2] = lo2(v2); v1[2] = hi2(v2);
                        v0[3] = lo2(v3); v1[3] = hi2(v3);
                        v0[4] = lo2(v4); v1[4] = hi2(v4);
                        v0[5] = lo2(ds2); v1[5] = hi2(ds2);
                        v0[6] = lo2(v6); v1[6] = hi2(v6);
                        v0[7] = lo2(v7); v1[7] = hi2(v7);
                        v0[8] = lo2(v8); v1[8] = hi2(v8);
                    }
                }
                emit_splat(g9, s_k[2 * p], c0, v0, lane);
                emit_splat(g9, s_k[2 * p + 1], c1, v1, lane);
            }
        }
    }
    if (STATS) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            n_sq += __shfl_xor_sync(0xffffffffu, n_sq, o);
            n_on += __shfl_xor_sync(0xffffffffu, n_on, o);
        }
        if (lane == 0) {
            atomicAdd(stats, n_sq);
            atomicAdd(stats + 1, n_on);
        }
    }
}

// ---------------------------------------------------------------------------
// TMA-staged warp tiles (variant 9): the arithmetic of variant 7 (one-warp
// tiles, PPT 1, batches of 32), with each batch of a tile's list staged in
// shared memory by one 1-D bulk copy (cp.async.bulk) of the records in list
// order, written after the sort by k_list_records.  Two buffers per warp: the
// next batch lands while the current one is composited.  Every wait on a copy
// is bounded: a warp whose copy does not arrive latches GS_ERR_TIMEOUT, lets
// its copies in flight land and stops.

__global__ void k_list_records(const uint32_t *__restrict__ svals, const int *n_keys_p, int64_t kcap,
                               const float4 *__restrict__ rec0, const float4 *__restrict__ rec1,
                               const float4 *__restrict__ rec2, uint32_t cap, float4 *__restrict__ lrec)
{
    const int64_t nk = min((int64_t)*n_keys_p, kcap);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nk; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = svals[j];
        float4 a = make_float4(0.f, 0.f, -1.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f), c = b;
        if (k < cap) {                      // else an empty splat (never for a consistent list)
            a = rec0[k];
            b = rec1[k];
            c = rec2[k];
            c.w = __uint_as_float(k);
        }
        lrec[3 * j] = a;
        lrec[3 * j + 1] = b;
        lrec[3 * j + 2] = c;
    }
}

template <int BATCH> struct TmaStage {
    float4 (*buf)[3 * BATCH];
    uint64_t *bar;
    uint32_t ph;            // phase parity of each buffer's barrier (bit s)
    int lane;
    uint32_t limit;         // polls of the next wait: the job's first-wait limit, then CULL_WAIT_LIMIT
    __device__ __forceinline__ void issue(const float4 *lrec, uint32_t b0, int cnt, int s)
    {
        if (lane == 0) {
            // generic-proxy reads of this buffer (the warp is past them) before the async-proxy write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[s], (uint32_t)cnt * 48u);
            bulk_g2s(buf[s], lrec + 3 * (size_t)b0, (uint32_t)cnt * 48u, &bar[s]);
        }
    }
    // wait for buffer s's copy; false (for the whole warp) if a lane's wait gave up
    __device__ __forceinline__ bool wait(int s)
    {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[s], (ph >> s) & 1u, limit));
        limit = CULL_WAIT_LIMIT;
        ph ^= 1u << s;
        return ok;
    }
};

template <int BATCH, int NW>
__global__ void __launch_bounds__(32 * NW, 5) k_raster_fwd_tma(const RasterJob J, const DevArgs *__restrict__ args,
                                                               int use_target, float *__restrict__ loss)
{
    __shared__ __align__(128) float4 buf_[NW][2][3 * BATCH];
    __shared__ __align__(8) uint64_t bar_[NW][2];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TmaStage<BATCH> S{buf_[wid], bar_[wid], 0u, lane, J.first_wait};
    if (lane == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    bool dead = false;
    float loss_part = 0.f;
    int view, tile;
    while (!dead && next_item<true>(J, &s_item, view, tile)) {
        float *__restrict__ image = J.image[view], *__restrict__ cfinal = J.cfinal[view];
        float *__restrict__ dimage = J.dimage[view];
        const DevCam &cam = args->cam[J.cam0 + view];
        const float *target = use_target ? args->target[J.cam0 + view] : nullptr;
        const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
        const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
        const int x = tx0 + lane % tw, y = ty0 + lane / tw;
        const float px = (float)x + 0.5f, pyv = (float)y + 0.5f;
        const uint2 rg = J.ranges[view][tile];
        const float4 *lrec = J.lrec[view];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
        bool live = x < W && y < H;
        int s = 0;
        if (rg.x < rg.y) S.issue(lrec, rg.x, min(BATCH, (int)(rg.y - rg.x)), 0);
        for (uint32_t b = rg.x; b < rg.y; b += BATCH, s ^= 1) {
            const int cnt = min(BATCH, (int)(rg.y - b));
            if (!__any_sync(0xffffffffu, live)) {      // done early: the copy of this batch still lands
                S.wait(s);
                break;
            }
            const bool more = b + BATCH < rg.y;
            if (more) S.issue(lrec, b + BATCH, min(BATCH, (int)(rg.y - b - BATCH)), s ^ 1);
            if (!S.wait(s)) {
                latch(J.status, GS_ERR_TIMEOUT);
                if (more) mbar_wait_bounded(&S.bar[s ^ 1], (S.ph >> (s ^ 1)) & 1u, CULL_WAIT_LIMIT);
                dead = true;
                break;
            }
            const float4 *B = S.buf[s];
            for (int e = 0; e < cnt && live; e++) {
                const float4 r0 = B[3 * e];        // (the tile is the warp's: every listed square overlaps it)
                const float dx = __fsub_rn(r0.x, px);
                if (fabsf(dx) > r0.z) continue;
                const float4 r1 = B[3 * e + 1];
                float dy, G;
                bool cl;
                const float a = splat_alpha_nb(r0, r1, dx, pyv, dy, G, cl);
                if (a == 0.f) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
                if (Tn < T_STOP) {
                    live = false;
                    continue;
                }
                const float4 c = B[3 * e + 2];
                const float aT = __fmul_rn(a, T);
                C0 = __fmaf_rn(c.x, aT, C0);
                C1 = __fmaf_rn(c.y, aT, C1);
                C2 = __fmaf_rn(c.z, aT, C2);
                T = Tn;
            }
            __syncwarp();                                // buffer s is read; it may be refilled
        }
        if (dead) break;
        if (x < W && y < H) {
            const int64_t HW = (int64_t)W * H, pix = (int64_t)y * W + x;
            image[pix] = C0;
            image[HW + pix] = C1;
            image[2 * HW + pix] = C2;
            if (cfinal) {
                cfinal[pix] = C0;
                cfinal[HW + pix] = C1;
                cfinal[2 * HW + pix] = C2;
            }
            if (target) {
                const float inv = cam.loss_inv;
                float d0 = C0 - target[pix], d1 = C1 - target[HW + pix], d2 = C2 - target[2 * HW + pix];
                dimage[pix] = (d0 > 0.f ? inv : (d0 < 0.f ? -inv : 0.f));
                dimage[HW + pix] = (d1 > 0.f ? inv : (d1 < 0.f ? -inv : 0.f));
                dimage[2 * HW + pix] = (d2 > 0.f ? inv : (d2 < 0.f ? -inv : 0.f));
                loss_part += (fabsf(d0) + fabsf(d1) + fabsf(d2)) * inv;
            }
        }
    }
    if (use_target) {
#pragma unroll
        for (int o = 16; o; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
        if (lane == 0 && loss_part != 0.f) atomicAdd(loss, loss_part);
    }
}

template <int BATCH, int NW, bool STATS = false>
__global__ void __launch_bounds__(32 * NW) k_raster_bwd_tma(const RasterJob J, const DevArgs *__restrict__ args,
                                                           unsigned long long *stats = nullptr)
{
    __shared__ __align__(128) float4 buf_[NW][2][3 * BATCH];
    __shared__ __align__(8) uint64_t bar_[NW][2];
    __shared__ int s_item;
    unsigned long long n_sq = 0, n_on = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TmaStage<BATCH> S{buf_[wid], bar_[wid], 0u, lane, J.first_wait};
    if (lane == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    bool dead = false;
    int view, tile;
    while (!dead && next_item<true>(J, &s_item, view, tile)) {
        const float *__restrict__ cfinal = J.cfinal[view], *__restrict__ dimage = J.dimage[view];
        float *__restrict__ g9 = J.g9[view];
        const DevCam &cam = args->cam[J.cam0 + view];
        const int W = cam.width, H = cam.height, tw = cam.tile_w, th = cam.tile_h, tiles_x = cam.tiles_x;
        const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
        const int x = tx0 + lane % tw, y = ty0 + lane / tw;
        const float px = (float)x + 0.5f, pyv = (float)y + 0.5f;
        const uint2 rg = J.ranges[view][tile];
        const float4 *lrec = J.lrec[view];
        float T = 1.f, gF = 0.f, gA = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        bool live = x < W && y < H;
        if (live) {
            const int64_t HW = (int64_t)W * H, pix = (int64_t)y * W + x;
            g0 = dimage[pix];
            g1 = dimage[HW + pix];
            g2 = dimage[2 * HW + pix];
            gF = g0 * cfinal[pix] + g1 * cfinal[HW + pix] + g2 * cfinal[2 * HW + pix];
        }
        int s = 0;
        if (rg.x < rg.y) S.issue(lrec, rg.x, min(BATCH, (int)(rg.y - rg.x)), 0);
        for (uint32_t b = rg.x; b < rg.y; b += BATCH, s ^= 1) {
            const int cnt = min(BATCH, (int)(rg.y - b));
            if (!__any_sync(0xffffffffu, live)) {
                S.wait(s);
                break;
            }
            const bool more = b + BATCH < rg.y;
            if (more) S.issue(lrec, b + BATCH, min(BATCH, (int)(rg.y - b - BATCH)), s ^ 1);
            if (!S.wait(s)) {
                latch(J.status, GS_ERR_TIMEOUT);
                if (more) mbar_wait_bounded(&S.bar[s ^ 1], (S.ph >> (s ^ 1)) & 1u, CULL_WAIT_LIMIT);
                dead = true;
                break;
            }
            const float4 *B = S.buf[s];
            for (int e = 0; e < cnt; e++) {
                const float4 r0 = B[3 * e];        // (the tile is the warp's: every listed square overlaps it)
                const float dx = __fsub_rn(r0.x, px);
                float v[9];                        // set where contrib (read only there)
                bool contrib = false;
                const float4 r1 = B[3 * e + 1];
                if (live && fabsf(dx) <= r0.z) {
                    float dy, G;
                    bool cl;
                    const float a = splat_alpha_nb(r0, r1, dx, pyv, dy, G, cl);
                    if (STATS) n_sq += fabsf(dy) <= r0.z ? 1 : 0;
                    if (a != 0.f) {
                        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
                        if (Tn < T_STOP) {
                            live = false;
                        } else {
                            if (STATS) n_on++;
                            contrib = true;
                            const float4 c = B[3 * e + 2];
                            const float aT = __fmul_rn(a, T);
                            const float gc = __fmaf_rn(g2, c.z, __fmaf_rn(g1, c.y, __fmul_rn(g0, c.x)));
                            gA = __fmaf_rn(aT, gc, gA);
                            const float dLda = __fmaf_rn(T, gc, -__fdividef(__fsub_rn(gF, gA), __fsub_rn(1.f, a)));
                            v[6] = __fmul_rn(g0, aT);
                            v[7] = __fmul_rn(g1, aT);
                            v[8] = __fmul_rn(g2, aT);
                            // the 0.999 clamp has no derivative: ds = 0 there
                            const float ds = cl ? 0.f : __fmul_rn(-a, dLda);
                            v[5] = ds;
                            const float sdx = __fmul_rn(ds, dx), sdy = __fmul_rn(ds, dy);
                            v[0] = sdx;
                            v[1] = sdy;
                            v[2] = __fmul_rn(sdx, dx);
                            v[3] = __fmul_rn(sdx, dy);
                            v[4] = __fmul_rn(sdy, dy);
                            T = Tn;
                        }
                    }
                }
                emit_splat_sel(g9, __float_as_uint(B[3 * e + 2].w), contrib, v, lane);
            }
            __syncwarp();
        }
        if (dead) break;
    }
    if (STATS) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            n_sq += __shfl_xor_sync(0xffffffffu, n_sq, o);
            n_on += __shfl_xor_sync(0xffffffffu, n_on, o);
        }
        if (lane == 0) {
            atomicAdd(stats, n_sq);
            atomicAdd(stats + 1, n_on);
        }
    }
}

typedef void (*RasterFwdFn)(const RasterJob, const DevArgs *, int, float *);
typedef void (*RasterBwdFn)(const RasterJob, const DevArgs *, unsigned long long *);

// Variant v < 6: PPT = 1 << (v >> 1), BATCH = (v & 1) ? 256 : 128, one tile
// per block.  v = 6, 7: warp tiles (32-pixel tiles, PPT 1), 4 warps with
// batches of 64 or 8 warps with batches of 32 per block.
static RasterFwdFn fwd_variant(int v)
{
    switch (v) {
    case 0: return k_raster_fwd<1, 128>;
    case 1: return k_raster_fwd<1, 256>;
    case 2: return k_raster_fwd<2, 128>;
    case 3: return k_raster_fwd<2, 256>;
    case 4: return k_raster_fwd<4, 128>;
    case 5: return k_raster_fwd<4, 256>;
    case 6: return k_raster_fwd<1, 64, 4>;
    case 7: return k_raster_fwd<1, 32, 8>;
    case 8: return k_raster_fwd_pairs<32, 8>;
    default: return k_raster_fwd_tma<32, 8>;
    }
}

static RasterBwdFn bwd_variant(int v, bool stats)
{
    switch (v * 2 + (stats ? 1 : 0)) {
    case 0: return k_raster_bwd<1, 128, false>;
    case 1: return k_raster_bwd<1, 128, true>;
    case 2: return k_raster_bwd<1, 256, false>;
    case 3: return k_raster_bwd<1, 256, true>;
    case 4: return k_raster_bwd<2, 128, false>;
    case 5: return k_raster_bwd<2, 128, true>;
    case 6: return k_raster_bwd<2, 256, false>;
    case 7: return k_raster_bwd<2, 256, true>;
    case 8: return k_raster_bwd<4, 128, false>;
    case 9: return k_raster_bwd<4, 128, true>;
    case 10: return k_raster_bwd<4, 256, false>;
    case 11: return k_raster_bwd<4, 256, true>;
    case 12: return k_raster_bwd<1, 64, false, 4>;
    case 13: return k_raster_bwd<1, 64, true, 4>;
    case 14: return k_raster_bwd<1, 32, false, 8>;
    case 15: return k_raster_bwd<1, 32, true, 8>;
    case 16: return k_raster_bwd_pairs<32, 8, false>;
    case 17: return k_raster_bwd_pairs<32, 8, true>;
    case 18: return k_raster_bwd_tma<32, 8, false>;
    default: return k_raster_bwd_tma<32, 8, true>;
    }
}

// Warps per block of a warp-tile variant, else 0.
static int warp_tile_warps(int v) { return v == 6 ? 4 : (v == 7 || v == 8 || v == 9) ? 8 : 0; }

bool raster_variant_ok(int v, int tile_w, int tile_h, bool has_records)
{
    if (v < 0 || v >= N_RASTER_VARIANTS) return false;
    if (v == RASTER_TMA_VARIANT && !has_records) return false;
    if (warp_tile_warps(v)) return tile_w * tile_h == 32;
    const int ppt = 1 << (v >> 1);
    const int threads = tile_w * tile_h / ppt;
    return tile_h % ppt == 0 && threads >= 32 && threads <= 256 && threads % 32 == 0;
}

// ---------------------------------------------------------------------------
// Chain rule of the projection (FP32 counterpart of the adjoint in §2.4 step 5).
// FIX = false: every visible Gaussian except those the gather flagged for the
// FP64 chain; FIX = true: the flagged ones, with the adjoint of the 2D
// covariance in FP64.
template <bool FIX, int DEG>
__global__ void __launch_bounds__(PROJ_BLOCK) k_project_bwd(const float *__restrict__ compact, int cap,
                                                            const int *n_vis_p, const DevArgs *__restrict__ args, int view,
                                                            const float *__restrict__ g9, float *__restrict__ grad,
                                                            int64_t gcap, const int32_t *__restrict__ ids,
                                                            const uint32_t *__restrict__ rmask,
                                                            const uint32_t *__restrict__ rprefix, const PrevMasks prev,
                                                            int *status, const int *__restrict__ n_fix,
                                                            const int32_t *__restrict__ fix_idx,
                                                            const uint8_t *__restrict__ fix_flag)
{
    __shared__ DevCam s_cam;
    if (threadIdx.x < sizeof(DevCam) / 4)
        ((uint32_t *)&s_cam)[threadIdx.x] = ((const uint32_t *)&args->cam[view])[threadIdx.x];
    __syncthreads();
    const int n_vis = min(*n_vis_p, cap);
    constexpr int deg = DEG, nk = (DEG + 1) * (DEG + 1);   // compile-time: Y and h stay in registers
    const DevCam &cam = s_cam;
    const int n_items = FIX ? min(*n_fix, n_vis) : n_vis;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_items; j += gridDim.x * blockDim.x) {
        const int k = FIX ? fix_idx[j] : j;
        // the splat's loads are issued before the flag that may skip it arrives
        float g[N_GEO];
#pragma unroll
        for (int r = 0; r < N_GEO; r++) g[r] = compact[r * (int64_t)cap + k];
        float gs[9];
        {
            const float4 *row = reinterpret_cast<const float4 *>(g9 + (int64_t)k * G9_STRIDE);
            const float4 a = row[0], b = row[1];
            gs[0] = a.x; gs[1] = a.y; gs[2] = a.z; gs[3] = a.w;
            gs[4] = b.x; gs[5] = b.y; gs[6] = b.z; gs[7] = b.w;
            gs[8] = g9[(int64_t)k * G9_STRIDE + 8];
        }
        if (!FIX && fix_flag[k]) continue;
        int64_t kk = k;
        bool accumulate = false;                   // an earlier view of the step wrote this row
        if (rmask) {
            int64_t i = ids[k];
            if (i < 0) continue;
            uint32_t word = rmask[i >> 5];
            kk = rprefix[i >> 5] + __popc(word & ((1u << (i & 31)) - 1u));
#pragma unroll
            for (int p = 0; p < MAX_VIEWS; p++)        // constant indices: the masks stay kernel parameters
                if (p < prev.n) accumulate |= ((prev.m[p][i >> 5] >> (i & 31)) & 1u) != 0u;
        }
        if (kk >= gcap) {          // the caller's gradient buffer is smaller than the visible set
            latch(status, GS_ERR_CAPACITY);
            continue;
        }
        Proj P;
        project_gaussian<FIX>(g, cam, P);   // as in the forward (FIX: the FP64 chain)
        if (P.keep) {
            // the rasterizer's sums (ds dx, ds dy, ds dx^2, ds dx dy, ds dy^2) over the splat's pixels, with
            // ds = -alpha dL/dalpha: the mean gradient is the conic times the first two, and sigma takes half
            // of A dx^2 and of C dy^2
            const float s0 = gs[0], s1 = gs[1];
            gs[0] = P.conA * s0 + P.conB * s1;
            gs[1] = P.conB * s0 + P.conC * s1;
            gs[2] = 0.5f * gs[2];
            gs[4] = 0.5f * gs[4];
        }
        float out[N_GEO];
#pragma unroll
        for (int r = 0; r < N_GEO; r++) out[r] = 0.f;
        bool ok = P.keep != 0;
        // ---- colour: SH coefficients and the viewing direction
        float vx = g[0] - cam.campos[0], vy = g[1] - cam.campos[1], vz = g[2] - cam.campos[2];
        float vn = sqrtf(vx * vx + vy * vy + vz * vz), ivn = 1.f / vn;
        float dir[3] = {vx * ivn, vy * ivn, vz * ivn};
        float Y[16];
        sh_basis(deg, dir[0], dir[1], dir[2], Y);
        float raw[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < nk; q++)
#pragma unroll
            for (int c = 0; c < 3; c++) raw[c] += Y[q] * compact[(N_GEO + 3 * q + c) * (int64_t)cap + k];
        float grgb[3];
#pragma unroll
        for (int c = 0; c < 3; c++) grgb[c] = (ok && raw[c] + 0.5f >= 0.f) ? gs[6 + c] : 0.f;
        float h[16];
#pragma unroll
        for (int q = 0; q < nk; q++) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float coef = compact[(N_GEO + 3 * q + c) * (int64_t)cap + k];
                acc += grgb[c] * coef;
                float gv = Y[q] * grgb[c];
                float *dst = grad + (N_GEO + 3 * q + c) * gcap + kk;
                if (accumulate) *dst += gv; else *dst = gv;
            }
            h[q] = acc;
        }
        float gdir[3];
        sh_basis_vjp(deg, dir[0], dir[1], dir[2], h, gdir);
        float dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        float gmu[3] = {(gdir[0] - dir[0] * dd) * ivn, (gdir[1] - dir[1] * dd) * ivn, (gdir[2] - dir[2] * dd) * ivn};
        if (ok) {
            // ---- opacity logit
            float o = 1.f / (1.f + expf(-g[ROW_OPAC]));
            // dL/do = sum G dL/dalpha = -(sum ds) / o (alpha = o G where it is not clamped; clamped pixels add
            // to neither sum), times do/dlogit = o (1 - o)
            out[ROW_OPAC] = -gs[5] * (1.f - o);
            float gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
            const float *R = cam.R;
            float pxc = P.p[0], pyc = P.p[1], pz = P.p[2];
            float iz = 1.f / pz, iz2 = iz * iz;
            float fx = cam.fx, fy = cam.fy;
            if (FIX) {
                Geo10 G;
#pragma unroll
                for (int k = 0; k < 10; k++) G.v[k] = g[k];
                const CovGrad cg = cov_chain_bwd_fp64(G, cam, gs[2], gs[3], gs[4]);
                gp0 = cg.gp[0]; gp1 = cg.gp[1]; gp2 = cg.gp[2];
#pragma unroll
                for (int k = 0; k < 3; k++) out[ROW_LS + k] = cg.gls[k];
#pragma unroll
                for (int k = 0; k < 4; k++) out[ROW_QUAT + k] = cg.gq[k];
            } else {
                // ---- conic -> covariance (a, b, c)
                float a = P.a, b = P.b, c = P.c;
                float id2 = 1.f / (P.det * P.det);
                float gA = gs[2], gB = gs[3], gC = gs[4];
                float ga = (-c * c * gA + b * c * gB - b * b * gC) * id2;
                float gb = (2.f * b * c * gA - (a * c + b * b) * gB + 2.f * a * b * gC) * id2;
                float gc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
                float hb = 0.5f * gb;
                // ---- Sigma2 = T Sigma3 T^T + 0.3 I
                const float *T = P.T;
                // gS3 = ga t0 t0^T + hb (t0 t1^T + t1 t0^T) + gc t1 t1^T (symmetric)
                float gS[9];
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int q = 0; q < 3; q++)
                        gS[r * 3 + q] = ga * T[r] * T[q] + hb * (T[r] * T[3 + q] + T[3 + r] * T[q]) + gc * T[3 + r] * T[3 + q];
                // gT = 2 G2 T Sigma3
                float S3f[9] = {P.S3[0], P.S3[1], P.S3[2], P.S3[1], P.S3[3], P.S3[4], P.S3[2], P.S3[4], P.S3[5]};
                float e0[3], e1[3];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    e0[q] = 2.f * (ga * T[q] + hb * T[3 + q]);
                    e1[q] = 2.f * (hb * T[q] + gc * T[3 + q]);
                }
                float gT[6];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    gT[q] = e0[0] * S3f[0 * 3 + q] + e0[1] * S3f[1 * 3 + q] + e0[2] * S3f[2 * 3 + q];
                    gT[3 + q] = e1[0] * S3f[0 * 3 + q] + e1[1] * S3f[1 * 3 + q] + e1[2] * S3f[2 * 3 + q];
                }
                // gJ = gT W^T (entries 00, 02, 11, 12)
                float gJ00 = gT[0] * R[0] + gT[1] * R[1] + gT[2] * R[2];
                float gJ02 = gT[0] * R[6] + gT[1] * R[7] + gT[2] * R[8];
                float gJ11 = gT[3] * R[3] + gT[4] * R[4] + gT[5] * R[5];
                float gJ12 = gT[3] * R[6] + gT[4] * R[7] + gT[5] * R[8];
                float iz3 = iz2 * iz;
                gp2 += -(gJ00 * fx + gJ11 * fy) * iz2;
                if (!P.cu) {
                    gp0 += -gJ02 * fx * iz2;
                    gp2 += 2.f * gJ02 * fx * pxc * iz3;
                } else {
                    float lim = pxc > 0.f ? cam.limx : -cam.limx;
                    gp2 += gJ02 * fx * lim * iz2;
                }
                if (!P.cw) {
                    gp1 += -gJ12 * fy * iz2;
                    gp2 += 2.f * gJ12 * fy * pyc * iz3;
                } else {
                    float lim = pyc > 0.f ? cam.limy : -cam.limy;
                    gp2 += gJ12 * fy * lim * iz2;
                }
                // Sigma3 = M M^T, M = Rq diag(s): gM = 2 gS M
                float M[9];
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int q = 0; q < 3; q++) M[r * 3 + q] = P.Rq[r * 3 + q] * P.s[q];
                float gR[9];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    float gsc = 0.f;
#pragma unroll
                    for (int r = 0; r < 3; r++) {
                        float gm = 2.f * (gS[r * 3 + 0] * M[0 * 3 + q] + gS[r * 3 + 1] * M[1 * 3 + q] + gS[r * 3 + 2] * M[2 * 3 + q]);
                        gsc += gm * P.Rq[r * 3 + q];
                        gR[r * 3 + q] = gm * P.s[q];
                    }
                    out[ROW_LS + q] = gsc * P.s[q];
                }
                // rotation -> normalised quaternion -> quaternion
                float qw = P.qh[0], qx = P.qh[1], qy = P.qh[2], qz = P.qh[3];
                float gw = -2.f * qz * gR[1] + 2.f * qy * gR[2] + 2.f * qz * gR[3] - 2.f * qx * gR[5] - 2.f * qy * gR[6] + 2.f * qx * gR[7];
                float gx = 2.f * qy * gR[1] + 2.f * qz * gR[2] + 2.f * qy * gR[3] - 4.f * qx * gR[4] - 2.f * qw * gR[5] + 2.f * qz * gR[6] + 2.f * qw * gR[7] - 4.f * qx * gR[8];
                float gy = -4.f * qy * gR[0] + 2.f * qx * gR[1] + 2.f * qw * gR[2] + 2.f * qx * gR[3] + 2.f * qz * gR[5] - 2.f * qw * gR[6] + 2.f * qz * gR[7] - 4.f * qy * gR[8];
                float gz = -4.f * qz * gR[0] - 2.f * qw * gR[1] + 2.f * qx * gR[2] + 2.f * qw * gR[3] - 4.f * qz * gR[4] + 2.f * qy * gR[5] + 2.f * qx * gR[6] + 2.f * qy * gR[7];
                float dq = gw * qw + gx * qx + gy * qy + gz * qz;
                float iqn = 1.f / P.qn;
                out[ROW_QUAT + 0] = (gw - qw * dq) * iqn;
                out[ROW_QUAT + 1] = (gx - qx * dq) * iqn;
                out[ROW_QUAT + 2] = (gy - qy * dq) * iqn;
                out[ROW_QUAT + 3] = (gz - qz * dq) * iqn;
            }
            // mean2d
            gp0 += gs[0] * fx * iz;
            gp1 += gs[1] * fy * iz;
            gp2 += -(gs[0] * fx * pxc + gs[1] * fy * pyc) * iz2;
            // p = W mu + t
            gmu[0] += R[0] * gp0 + R[3] * gp1 + R[6] * gp2;
            gmu[1] += R[1] * gp0 + R[4] * gp1 + R[7] * gp2;
            gmu[2] += R[2] * gp0 + R[5] * gp1 + R[8] * gp2;
        }
        out[0] = ok ? gmu[0] : 0.f;
        out[1] = ok ? gmu[1] : 0.f;
        out[2] = ok ? gmu[2] : 0.f;
#pragma unroll
        for (int r = 0; r < N_GEO; r++) {
            float *dst = grad + r * gcap + kk;
            if (accumulate) *dst += out[r]; else *dst = out[r];
        }
    }
}

// ---------------------------------------------------------------------------
// Zero rows x n entries (n = min(*n_dev, cap)) of a [rows][pitch] array, or,
// with aos, the first n records of `rows` floats each.
__global__ void k_zero_rows(float *buf, int rows, int64_t pitch, const int *n_dev, int cap, int aos)
{
    int n = n_dev ? min(*n_dev, cap) : cap;
    int64_t total = (int64_t)rows * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        if (aos) {
            buf[e] = 0.f;
        } else {
            int64_t r = e / n, k = e - r * n;
            buf[r * pitch + k] = 0.f;
        }
    }
}

void launch_zero_rows(float *buf, int rows, int64_t pitch, const int *n_dev, int cap, Work &w, cudaStream_t s,
                      bool aos)
{
    k_zero_rows<<<w.grid((int64_t)rows * cap, 256), 256, 0, s>>>(buf, rows, pitch, n_dev, cap, aos ? 1 : 0);
}

__global__ void k_loss_l1(const float *__restrict__ image, const float *__restrict__ target, int64_t count,
                          float *loss, float *dimage)
{
    __shared__ float s_red[32];
    float inv = 1.f / (float)count, part = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        float d = image[e] - target[e];
        part += fabsf(d);
        if (dimage) dimage[e] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    float t = block_sum(part * inv, s_red);
    if (threadIdx.x == 0) atomicAdd(loss, t);
}

void launch_loss_l1(const float *image, const float *target, int64_t count, float *loss, float *dimage, Work &w,
                    cudaStream_t s)
{
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    k_loss_l1<<<w.grid(count, 256, 4), 256, 0, s>>>(image, target, count, loss, dimage);
}

void prepare_view(const SceneView &sc, const DevArgs *args, int view, const int32_t *ids, const int *n_vis,
                  RenderBufs &rb, const DevCam &cam, Work &w, cudaStream_t s, bool zero_g9)
{
    const int cap = (int)rb.cap;
    decltype(&k_gather_project<0, float, GS_OPT_ADAM>) gp = nullptr;
    with_opt(sc.opt, [&](auto o) {
        constexpr int O = decltype(o)::value;
        gp = sc.prec == GS_FP32
                 ? (sc.deg == 3 ? k_gather_project<3, float, O> : sc.deg == 2 ? k_gather_project<2, float, O>
                    : sc.deg == 1 ? k_gather_project<1, float, O> : k_gather_project<0, float, O>)
                 : (sc.deg == 3 ? k_gather_project<3, __nv_bfloat16, O>
                    : sc.deg == 2 ? k_gather_project<2, __nv_bfloat16, O>
                    : sc.deg == 1 ? k_gather_project<1, __nv_bfloat16, O> : k_gather_project<0, __nv_bfloat16, O>);
    });
    const int tiles = cam.tiles_x * cam.tiles_y;
    cudaMemsetAsync(rb.n_fix, 0, sizeof(int), s);
    cudaMemsetAsync(rb.n_big, 0, 3 * sizeof(int), s);
    // gather and projection
    gp<<<w.grid(cap, PROJ_BLOCK, 12), PROJ_BLOCK, 0, s>>>(sc, ids, n_vis, cap, args, view, rb.compact, rb.rec0, rb.rec1,
                                                          rb.rec2, rb.depth, rb.rect, rb.n_fix, rb.fix_idx,
                                                          rb.fix_flag, rb.n_big, rb.big_idx);
    // the FP64 fix-ups beside the counting of the other splats' keys (which
    // skips the flagged ones); the big-rectangle counts wait for them
    const cudaStream_t fs = w.fork(s);
    k_fix_project<<<w.num_sms, PROJ_BLOCK, 0, fs>>>(rb.compact, cap, rb.n_fix, rb.fix_idx, args, view, rb.rec0, rb.rec1,
                                                     rb.rect, rb.n_big, rb.big_idx);
    if (zero_g9) launch_zero_rows(rb.g9, G9_STRIDE, cap, n_vis, cap, w, fs, true);
    w.side_done(fs);
    build_tile_lists(args, view, n_vis, rb, tiles, w, s);
    rb.sorted_keys = rb.tk[1];
    rb.sorted_vals = rb.tv[1];
    rb.tiles = tiles;

}

static RasterJob make_job(int n_views, RenderBufs *const *rbs, int *work)
{
    RasterJob J{};
    J.n_views = n_views;
    J.tile_ofs[0] = 0;
    for (int v = 0; v < n_views; v++) {
        const RenderBufs &rb = *rbs[v];
        J.tile_ofs[v + 1] = J.tile_ofs[v] + rb.tiles;
        J.ranges[v] = rb.ranges;
        J.svals[v] = rb.sorted_vals;
        J.rec0[v] = rb.rec0;
        J.rec1[v] = rb.rec1;
        J.rec2[v] = rb.rec2;
        J.cfinal[v] = rb.cfinal;
        J.g9[v] = rb.g9;
        J.cap[v] = (uint32_t)rb.cap;
        J.lrec[v] = rb.lrec;
        J.first_tiles[v] = rb.first_tiles;
        J.n_first[v] = rb.n_big + 2;
    }
    J.work = work;
    return J;
}

// Launch shape of variant v: persistent blocks, enough to fill the GPU and
// never more than the items (warp tiles: an item per warp).
struct RasterShape {
    int grid, block;
};
static RasterShape raster_shape(int v, int items, int tile_w, int tile_h, const Work &w)
{
    const int nw = warp_tile_warps(v);
    if (nw) return {std::max(1, std::min((items + nw - 1) / nw, w.num_sms * 64 / nw)), 32 * nw};
    const int ppt = 1 << (v >> 1);
    return {std::max(1, std::min(items, w.num_sms * 32)), tile_w * tile_h / ppt};
}

// The list-order records of a view, written by the first rasterizer pass that
// stages from them (the forward when it is variant 9, else the backward), so
// their cost counts toward the variant that uses them.
static void list_records(RenderBufs &rb, Work &w, cudaStream_t s)
{
    if (!rb.lrec) return;
    k_list_records<<<w.grid(rb.kcap, 256, 8), 256, 0, s>>>(rb.sorted_vals, rb.n_keys, rb.kcap, rb.rec0, rb.rec1, rb.rec2,
                                                          (uint32_t)rb.cap, rb.lrec);
}

void raster_forward(const DevArgs *args, int n_views, RenderBufs *const *rbs, const DevCam *cams, float *const *images,
                    bool use_target, float *const *dimages, float *loss, int *work, Work &w, cudaStream_t s, int cam0)
{
    if (rbs[0]->variant == RASTER_TMA_VARIANT)
        for (int v = 0; v < n_views; v++) list_records(*rbs[v], w, s);
    RasterJob J = make_job(n_views, rbs, work);
    J.cam0 = cam0;
    J.status = w.status;
    J.first_wait = w.cull_first_wait;
    for (int v = 0; v < n_views; v++) {
        J.image[v] = images[v];
        if (images[v] == rbs[v]->cfinal) J.cfinal[v] = nullptr;
        J.dimage[v] = use_target ? dimages[v] : nullptr;
    }
    const RenderBufs &rb0 = *rbs[0];
    const RasterShape sh = raster_shape(rb0.variant, J.tile_ofs[n_views], cams[0].tile_w, cams[0].tile_h, w);
    cudaMemsetAsync(work, 0, sizeof(int), s);
    fwd_variant(rb0.variant)<<<sh.grid, sh.block, 0, s>>>(J, args, use_target ? 1 : 0, loss);
}

// A job over one view of the argument block: slots 0..view, only `view` with items.
static RasterJob single_view_job(int view, RenderBufs &rb, int *work)
{
    RenderBufs *rbs[MAX_VIEWS] = {nullptr};
    for (int v = 0; v <= view; v++) rbs[v] = &rb;
    RasterJob J = make_job(view + 1, rbs, work);
    for (int v = 0; v <= view; v++) {
        J.tile_ofs[v + 1] = v < view ? 0 : rb.tiles;
        if (v < view) J.n_first[v] = nullptr;
    }
    return J;
}

void render_forward(const SceneView &sc, const DevArgs *args, int view, const int32_t *ids, const int *n_vis,
                    RenderBufs &rb, const DevCam &cam, float *image, bool use_target, float *dimage, float *loss,
                    Work &w, cudaStream_t s, int *work)
{
    prepare_view(sc, args, view, ids, n_vis, rb, cam, w, s);
    if (rb.variant == RASTER_TMA_VARIANT) list_records(rb, w, s);
    RasterJob J = single_view_job(view, rb, work);
    J.status = w.status;
    J.first_wait = w.cull_first_wait;
    for (int v = 0; v <= view; v++) {
        J.image[v] = image;
        J.cfinal[v] = image == rb.cfinal ? nullptr : rb.cfinal;
        J.dimage[v] = use_target ? dimage : nullptr;
    }
    const RasterShape sh = raster_shape(rb.variant, rb.tiles, cam.tile_w, cam.tile_h, w);
    cudaMemsetAsync(work, 0, sizeof(int), s);
    fwd_variant(rb.variant)<<<sh.grid, sh.block, 0, s>>>(J, args, use_target ? 1 : 0, loss);
}

void raster_backward(const DevArgs *args, int n_views, RenderBufs *const *rbs, const DevCam *cams,
                     const float *const *dimages, const int *const *n_vis, int *work, Work &w, cudaStream_t s,
                     unsigned long long *stats, int cam0, bool g9_zeroed)
{
    if (rbs[0]->variant_bwd == RASTER_TMA_VARIANT && rbs[0]->variant != RASTER_TMA_VARIANT)
        for (int v = 0; v < n_views; v++) list_records(*rbs[v], w, s);
    for (int v = 0; v < n_views && !g9_zeroed; v++) {
        const int cap = (int)rbs[v]->cap;
        launch_zero_rows(rbs[v]->g9, G9_STRIDE, cap, n_vis[v], cap, w, s, true);
    }
    RasterJob J = make_job(n_views, rbs, work);
    J.cam0 = cam0;
    J.status = w.status;
    J.first_wait = w.cull_first_wait;
    for (int v = 0; v < n_views; v++) J.dimage[v] = const_cast<float *>(dimages[v]);
    const RenderBufs &rb0 = *rbs[0];
    const RasterShape sh = raster_shape(rb0.variant_bwd, J.tile_ofs[n_views], cams[0].tile_w, cams[0].tile_h, w);
    cudaMemsetAsync(work, 0, sizeof(int), s);
    w.mark(TP_RBWD0, s);
    bwd_variant(rb0.variant_bwd, stats != nullptr)<<<sh.grid, sh.block, 0, s>>>(J, args, stats);
    w.mark(TP_RBWD1, s);
}

typedef void (*ProjBwdFn)(const float *, int, const int *, const DevArgs *, int, const float *, float *, int64_t,
                          const int32_t *, const uint32_t *, const uint32_t *, const PrevMasks, int *, const int *,
                          const int32_t *, const uint8_t *);

template <bool FIX> static ProjBwdFn pbwd_for(int deg)
{
    switch (deg) {
    case 0: return k_project_bwd<FIX, 0>;
    case 1: return k_project_bwd<FIX, 1>;
    case 2: return k_project_bwd<FIX, 2>;
    default: return k_project_bwd<FIX, 3>;
    }
}

void project_backward(const SceneView &sc, const DevArgs *args, int view, const int *n_vis, RenderBufs &rb,
                      float *grad, int64_t gcap, const uint32_t *remap_mask, const uint32_t *remap_prefix,
                      const int32_t *ids, const PrevMasks &prev, Work &w, cudaStream_t s)
{
    const int cap = (int)rb.cap;
    // the FP64 adjoint of the flagged splats beside the FP32 one of the others
    // (each Gaussian's rows are written by exactly one of the two)
    const cudaStream_t fs = w.fork(s);
    pbwd_for<true>(sc.deg)<<<w.num_sms, PROJ_BLOCK, 0, fs>>>(
        rb.compact, cap, n_vis, args, view, rb.g9, grad, gcap, ids, remap_mask, remap_prefix, prev,
        w.status, rb.n_fix, rb.fix_idx, rb.fix_flag);
    w.side_done(fs);
    pbwd_for<false>(sc.deg)<<<w.grid(cap, PROJ_BLOCK, 12), PROJ_BLOCK, 0, s>>>(
        rb.compact, cap, n_vis, args, view, rb.g9, grad, gcap, ids, remap_mask, remap_prefix, prev,
        w.status, rb.n_fix, rb.fix_idx, rb.fix_flag);
    w.wait_side(s);
}

void render_backward(const SceneView &sc, const DevArgs *args, int view, const int *n_vis, RenderBufs &rb,
                     const DevCam &cam, const float *dimage, float *grad, int64_t gcap, const uint32_t *remap_mask,
                     const uint32_t *remap_prefix, const int32_t *ids, Work &w, cudaStream_t s,
                     int *work, unsigned long long *stats)
{
    const int cap = (int)rb.cap;
    if (rb.variant_bwd == RASTER_TMA_VARIANT && rb.variant != RASTER_TMA_VARIANT) list_records(rb, w, s);
    launch_zero_rows(rb.g9, G9_STRIDE, cap, n_vis, cap, w, s, true);
    RasterJob J = single_view_job(view, rb, work);
    J.status = w.status;
    J.first_wait = w.cull_first_wait;
    for (int v = 0; v <= view; v++) J.dimage[v] = const_cast<float *>(dimage);
    const RasterShape sh = raster_shape(rb.variant_bwd, rb.tiles, cam.tile_w, cam.tile_h, w);
    cudaMemsetAsync(work, 0, sizeof(int), s);
    if (view == 0) w.mark(TP_RBWD0, s);
    bwd_variant(rb.variant_bwd, stats != nullptr)<<<sh.grid, sh.block, 0, s>>>(J, args, stats);
    if (view == 0) w.mark(TP_RBWD1, s);
    project_backward(sc, args, view, n_vis, rb, grad, gcap, remap_mask, remap_prefix, ids, PrevMasks{}, w, s);
}

}  // namespace gs
