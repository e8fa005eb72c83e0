// k_lists.cu -- each view's per-tile lists of the splats that can reach the
// tile, in front-to-back order (§2.4 step 2, tile binning and sort):
//
//   k_tiles_count, k_big_counts          the tiles each splat reaches (the
//                                        list filter): a count per tile
//   scan_counts                          each tile's first key, the key total
//   k_tiles_emit, k_big_emit             (depth, splat) keys into the tiles'
//                                        lists through per-tile cursors
//   k_find_long                          the long lists (and those the
//                                        rasterizers take first)
//   k_tile_sort(_long)                   each list sorted by depth (ties by
//                                        Gaussian id) with bitonic networks
#include "gs_kernels.cuh"

namespace gs {

// Can splat (r0, r1) reach alpha >= 1/255 at any pixel centre of the box
// [X0, X1] x [Y0, Y1]?  Intersects the box with the splat's square (widened
// by a small margin), takes the minimum of sigma over the remaining rectangle
// (zero if the mean is inside, otherwise on an edge, where sigma is a 1-D
// quadratic) and compares o exp(-sigma_min) with the floor, with 0.1% slack.
// It only ever says "no" when no pixel can pass the per-pixel tests, so
// dropping such splats leaves every pixel's result unchanged.
// Every operation is an explicitly rounded intrinsic (no contraction into FMAs
// that could differ between the kernels that inline it): the big list's key
// counting and key emission, in different kernels, must take the same
// decisions (the small rectangles' emission reads the count's masks).
__device__ __forceinline__ float q_sigma(float A, float B, float C, float dx, float dy)
{
    // 0.5 (A dx^2 + C dy^2) + B dx dy
    const float a = __fmul_rn(__fmul_rn(A, dx), dx), c = __fmul_rn(__fmul_rn(C, dy), dy);
    return __fadd_rn(__fmul_rn(0.5f, __fadd_rn(a, c)), __fmul_rn(__fmul_rn(B, dx), dy));
}

// The edge minimisers use the splat's ratios B / C and B / A (reach_ratios,
// formed once per splat); a minimiser off by a rounding raises the edge's
// minimum by a second-order amount, far inside the slack.
__device__ __forceinline__ float2 reach_ratios(float4 r1)
{
    return make_float2(__fdiv_rn(r1.y, r1.z), __fdiv_rn(r1.y, r1.x));
}

__device__ __forceinline__ bool splat_reaches_box(float4 r0, float4 r1, float2 bq, float X0, float X1, float Y0,
                                                  float Y1)
{
    const float margin = 1e-3f;
    const float ext = __fadd_rn(r0.z, margin);
    const float x0 = fmaxf(X0, __fsub_rn(r0.x, ext)), x1 = fminf(X1, __fadd_rn(r0.x, ext));
    const float y0 = fmaxf(Y0, __fsub_rn(r0.y, ext)), y1 = fminf(Y1, __fadd_rn(r0.y, ext));
    if (x0 > x1 || y0 > y1) return false;
    // d = mean - p over the rectangle
    const float dxl = __fsub_rn(r0.x, x1), dxh = __fsub_rn(r0.x, x0);
    const float dyl = __fsub_rn(r0.y, y1), dyh = __fsub_rn(r0.y, y0);
    const float A = r1.x, B = r1.y, C = r1.z;
    float smin = 0.f;
    if (!(dxl <= 0.f && dxh >= 0.f && dyl <= 0.f && dyh >= 0.f)) {
        smin = 3.4e38f;
        // edges dx = const: minimiser dy = -B dx / C
        const float dxs[2] = {dxl, dxh};
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float dx = dxs[k];
            const float dy = fminf(fmaxf(-__fmul_rn(bq.x, dx), dyl), dyh);
            smin = fminf(smin, q_sigma(A, B, C, dx, dy));
        }
        const float dys[2] = {dyl, dyh};
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const float dy = dys[k];
            const float dx = fminf(fmaxf(-__fmul_rn(bq.y, dy), dxl), dxh);
            smin = fminf(smin, q_sigma(A, B, C, dx, dy));
        }
        smin = fmaxf(smin, 0.f);
    }
    return __fmul_rn(r0.w, __expf(-smin)) >= ALPHA_MIN * 0.999f;
}

// Pixel-centre box of tile (t_x, t_y).
__device__ __forceinline__ void tile_box(const DevCam &cam, int t_x, int t_y, float &X0, float &X1, float &Y0,
                                         float &Y1)
{
    X0 = (float)(t_x * cam.tile_w) + 0.5f;
    X1 = X0 + (float)(cam.tile_w - 1);
    Y0 = (float)(t_y * cam.tile_h) + 0.5f;
    Y1 = Y0 + (float)(cam.tile_h - 1);
}


// Tiles reached by the splats of the big list (large rectangles, FP64-fixed
// splats): one warp per splat, lanes over the rectangle's tiles.
__global__ void k_big_counts(const float4 *__restrict__ rec0, const float4 *__restrict__ rec1,
                             const uint2 *__restrict__ rect, const int *__restrict__ n_big,
                             const int32_t *__restrict__ big_idx, int cap, const DevArgs *__restrict__ args, int view,
                             uint32_t *__restrict__ tile_cnt)
{
    const int nb = min(*n_big, cap);
    const DevCam &cam = args->cam[view];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nb; j += nwarps) {
        const int k = big_idx[j];
        const uint2 rc = rect[k];
        const int x0 = rc.x & 0xffff, x1 = rc.x >> 16, y0 = rc.y & 0xffff, y1 = rc.y >> 16;
        const int wdt = x1 - x0, cnt_all = wdt * (y1 - y0);
        if (cnt_all <= 0) continue;
        const float4 r0 = rec0[k], r1 = rec1[k];
        const float2 bq = reach_ratios(r1);
        for (int t = lane; t < cnt_all; t += 32) {
            const int tx = x0 + t % wdt, ty = y0 + t / wdt;
            float X0, X1, Y0, Y1;
            tile_box(cam, tx, ty, X0, X1, Y0, Y1);
            if (splat_reaches_box(r0, r1, bq, X0, X1, Y0, Y1)) atomicAdd(tile_cnt + ty * cam.tiles_x + tx, 1u);
        }
    }
}

// Row of pair j in a rectangle of width w as (j * ceil(2^16 / w)) >> 16:
// checked at compile time for every width and pair index a rectangle of at
// most BIG_RECT tiles has.
constexpr bool row_by_multiply_shift_exact(int max_area)
{
    for (int w = 1; w <= max_area; w++) {
        const uint32_t inv = (65536u + (uint32_t)w - 1u) / (uint32_t)w;
        for (int j = 0; j < max_area; j++)
            if ((int)(((uint32_t)j * inv) >> 16) != j / w) return false;
    }
    return true;
}
static_assert(row_by_multiply_shift_exact(BIG_RECT), "pair row index by multiply-shift is inexact at BIG_RECT");

// The small rectangles' (splat, tile) pairs, load-balanced over a warp: the
// warp takes 32 splats (kept, not FP64-flagged, at most BIG_RECT tiles: the
// partition k_gather_project leaves to it) and its lanes walk their
// concatenated pairs 32 at a time, so that the atomics of different pairs are
// in flight together.
//   k_tiles_count: every pair of a rectangle, through the list filter; one
//   more key for each tile reached, and each splat's reached tiles as a mask
//   (bit j: the j-th tile of its rectangle, row-major; BIG_RECT <= 32).
//   k_tiles_emit: only the reached pairs (the set bits of the masks), with no
//   filter; the key (depth, k) into the tile's list at slot tile_off[t] + (a
//   cursor of t), complete but unordered until k_tile_sort.
constexpr int TILES_BLOCK = 256;
static_assert(BIG_RECT <= 32, "a small rectangle's reached tiles fit one 32-bit mask");

// Exclusive and total sums of `area` over the warp, and the last lane whose
// pairs start at or before pair q of the concatenation.
__device__ __forceinline__ int warp_excl_scan(int area, int lane, int &total)
{
    int incl = area;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - area;
}
__device__ __forceinline__ int owner_lane(int ex, int q)
{
    int sl = 0;
#pragma unroll
    for (int st = 16; st; st >>= 1) {
        const int c = sl + st;
        if (__shfl_sync(0xffffffffu, ex, c) <= q) sl = c;
    }
    return sl;
}

__global__ void __launch_bounds__(TILES_BLOCK) k_tiles_count(const uint2 *__restrict__ rect,
                                                             const float4 *__restrict__ rec0,
                                                             const float4 *__restrict__ rec1,
                                                             const uint8_t *__restrict__ fix_flag, const int *n_vis_p,
                                                             int cap, const DevArgs *__restrict__ args, int view,
                                                             uint32_t *tile_cnt, uint32_t *__restrict__ reach)
{
    // the filter's results of one warp's concatenated pairs (at most 32 x 32)
    __shared__ uint32_t s_hit[TILES_BLOCK / 32][BIG_RECT + 1];
    const int n = min(*n_vis_p, cap);
    const DevCam &cam = args->cam[view];
    const int tiles_x = cam.tiles_x;
    const int lane = threadIdx.x & 31;
    uint32_t *hit = s_hit[threadIdx.x >> 5];
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * 32 < n; g += nwarps) {
        const int k = g * 32 + lane;
        uint2 rc = make_uint2(0u, 0u);
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        int area = 0;
        if (k < n && !fix_flag[k]) {
            rc = rect[k];
            area = (int)((rc.x >> 16) - (rc.x & 0xffff)) * (int)((rc.y >> 16) - (rc.y & 0xffff));
            if (area > 0 && area <= BIG_RECT) {
                r0 = rec0[k];
                r1 = rec1[k];
            } else {
                area = 0;
            }
        }
        const float2 bq = area ? reach_ratios(r1) : make_float2(0.f, 0.f);
        int total;
        const int ex = warp_excl_scan(area, lane, total);
        // j / width as (j * ceil(2^16 / width)) >> 16: exact for j * width < 2^16 (here j < 32, width <= 32)
        const int wd = area ? (int)((rc.x >> 16) - (rc.x & 0xffff)) : 1;
        const uint32_t inv = (65536u + (uint32_t)wd - 1u) / (uint32_t)wd;
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            const int sl = owner_lane(ex, q);
            const uint32_t rcx = __shfl_sync(0xffffffffu, rc.x, sl), rcy = __shfl_sync(0xffffffffu, rc.y, sl);
            const float4 a0 = make_float4(__shfl_sync(0xffffffffu, r0.x, sl), __shfl_sync(0xffffffffu, r0.y, sl),
                                          __shfl_sync(0xffffffffu, r0.z, sl), __shfl_sync(0xffffffffu, r0.w, sl));
            const float4 a1 = make_float4(__shfl_sync(0xffffffffu, r1.x, sl), __shfl_sync(0xffffffffu, r1.y, sl),
                                          __shfl_sync(0xffffffffu, r1.z, sl), 0.f);
            const float2 bqs = make_float2(__shfl_sync(0xffffffffu, bq.x, sl), __shfl_sync(0xffffffffu, bq.y, sl));
            const int exs = __shfl_sync(0xffffffffu, ex, sl);
            const uint32_t invs = __shfl_sync(0xffffffffu, inv, sl);
            bool reached = false;
            int t = 0;
            if (q < total) {
                const int x0 = (int)(rcx & 0xffff), wdt = (int)(rcx >> 16) - x0, y0 = (int)(rcy & 0xffff);
                const int j = q - exs, row = (int)(((uint32_t)j * invs) >> 16);
                const int tx = x0 + (j - row * wdt), ty = y0 + row;
                float X0, X1, Y0, Y1;
                tile_box(cam, tx, ty, X0, X1, Y0, Y1);
                reached = splat_reaches_box(a0, a1, bqs, X0, X1, Y0, Y1);
                t = ty * tiles_x + tx;
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, reached);
            if (lane == 0) hit[q0 >> 5] = bits;
            if (reached) atomicAdd(tile_cnt + t, 1u);
        }
        __syncwarp();
        // this lane's bits [ex, ex + area) of the concatenation
        uint32_t m = 0u;
        if (area) {
            const int w0 = ex >> 5, b0 = ex & 31;
            const uint32_t lo = hit[w0], hi = (b0 && w0 + 1 <= BIG_RECT) ? hit[w0 + 1] : 0u;
            m = __funnelshift_r(lo, hi, b0);
            if (area < 32) m &= (1u << area) - 1u;
        }
        if (k < n) reach[k] = m;
        __syncwarp();                                     // hit[] is read before the next group writes it
    }
}

__global__ void __launch_bounds__(TILES_BLOCK) k_tiles_emit(const uint2 *__restrict__ rect,
                                                            const uint32_t *__restrict__ reach,
                                                            const uint32_t *__restrict__ depth, const int *n_vis_p,
                                                            int cap, int64_t kcap, const DevArgs *__restrict__ args,
                                                            int view, const uint32_t *__restrict__ tile_off,
                                                            uint32_t *tile_cur, uint32_t *bkey, uint32_t *bval)
{
    const int n = min(*n_vis_p, cap);
    const DevCam &cam = args->cam[view];
    const int tiles_x = cam.tiles_x;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * 32 < n; g += nwarps) {
        const int k = g * 32 + lane;
        uint2 rc = make_uint2(0u, 0u);
        uint32_t m = 0u, dk = 0u;
        if (k < n) {
            m = reach[k];
            if (m) {
                rc = rect[k];
                dk = depth[k];
            }
        }
        int total;
        const int ex = warp_excl_scan(__popc(m), lane, total);
        const int wd = m ? (int)((rc.x >> 16) - (rc.x & 0xffff)) : 1;
        const uint32_t inv = (65536u + (uint32_t)wd - 1u) / (uint32_t)wd;
        for (int q0 = 0; q0 < total; q0 += 32) {
            const int q = q0 + lane;
            const int sl = owner_lane(ex, q);
            const uint32_t rcx = __shfl_sync(0xffffffffu, rc.x, sl), rcy = __shfl_sync(0xffffffffu, rc.y, sl);
            const uint32_t ms = __shfl_sync(0xffffffffu, m, sl), invs = __shfl_sync(0xffffffffu, inv, sl);
            const uint32_t dks = __shfl_sync(0xffffffffu, dk, sl);
            const int exs = __shfl_sync(0xffffffffu, ex, sl);
            if (q >= total) continue;
            const int j = (int)__fns(ms, 0u, q - exs + 1);         // the (q - exs)-th set bit: a tile of the rectangle
            const int x0 = (int)(rcx & 0xffff), wdt = (int)(rcx >> 16) - x0, y0 = (int)(rcy & 0xffff);
            const int row = (int)(((uint32_t)j * invs) >> 16);
            const int t = (y0 + row) * tiles_x + x0 + (j - row * wdt);
            const int64_t p = (int64_t)tile_off[t] + atomicAdd(tile_cur + t, 1u);
            if (p < kcap) {
                bkey[p] = dks;
                bval[p] = (uint32_t)(g * 32 + sl);
            }
        }
    }
}

// The keys of the big list: one warp per splat, lanes over its tiles.
__global__ void k_big_emit(const uint2 *__restrict__ rect, const float4 *__restrict__ rec0,
                           const float4 *__restrict__ rec1, const uint32_t *__restrict__ depth,
                           const int *__restrict__ n_big, const int32_t *__restrict__ big_idx, int cap, int64_t kcap,
                           const DevArgs *__restrict__ args, int view, const uint32_t *__restrict__ tile_off,
                           uint32_t *tile_cur, uint32_t *bkey, uint32_t *bval)
{
    const int nb = min(*n_big, cap);
    const DevCam &cam = args->cam[view];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nb; j += nwarps) {
        const int k = big_idx[j];
        const uint2 rc = rect[k];
        const int x0 = rc.x & 0xffff, x1 = rc.x >> 16, y0 = rc.y & 0xffff, y1 = rc.y >> 16;
        const int wdt = x1 - x0, cnt_all = wdt * (y1 - y0);
        if (cnt_all <= 0) continue;
        const float4 r0 = rec0[k], r1 = rec1[k];
        const float2 bq = reach_ratios(r1);
        const uint32_t dk = depth[k];
        for (int tt = lane; tt < cnt_all; tt += 32) {
            const int tx = x0 + tt % wdt, ty = y0 + tt / wdt;
            float X0, X1, Y0, Y1;
            tile_box(cam, tx, ty, X0, X1, Y0, Y1);
            if (!splat_reaches_box(r0, r1, bq, X0, X1, Y0, Y1)) continue;
            const int t = ty * cam.tiles_x + tx;
            const int64_t p = (int64_t)tile_off[t] + atomicAdd(tile_cur + t, 1u);
            if (p < kcap) {
                bkey[p] = dk;
                bval[p] = (uint32_t)k;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Per-tile sort of the lists into front-to-back order: by depth, ties by the
// splat's index (ascending ids: the visible set is compacted in id order), the
// order of one global sort on (tile, depth, id).  Keys are (depth bits << 32 |
// splat): depths are positive, so their bits order as unsigned integers.  All
// sorts are bitonic networks whose every comparator puts the minimum at the
// lower index (the first step of each merge compares mirrored positions), so
// a list padded with +inf needs no direction changes.

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a < b ? b : a; }

// N keys in a warp (N = 32, 64, 128 or 256): element e = 32 r + lane held in
// v[r].  Pairs within a row are exchanged through shuffles, pairs across rows
// stay in the lane's registers.
template <int N>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&v)[N / 32], int lane)
{
    constexpr int R = N / 32;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        // first step of the merge: e pairs with its mirror in the block of k
        if (k <= 32) {
            const bool lower = (lane & (k >> 1)) == 0;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const unsigned long long p = __shfl_xor_sync(0xffffffffu, v[r], k - 1);
                v[r] = lower ? umin64(v[r], p) : umax64(v[r], p);
            }
        } else {
            const int rm = (k >> 5) - 1;                  // mirror: row r ^ rm, lane ^ 31
            unsigned long long p[R];
#pragma unroll
            for (int r = 0; r < R; r++) p[r] = __shfl_xor_sync(0xffffffffu, v[r ^ rm], 31);
#pragma unroll
            for (int r = 0; r < R; r++) {
                // the lower element of the pair is the one in the lower half of the block of k
                const bool lower = ((r * 32) & (k >> 1)) == 0;
                v[r] = lower ? umin64(v[r], p[r]) : umax64(v[r], p[r]);
            }
        }
        // then pairs at distance j = k/4, ..., 1
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < R; r++)
                    if ((r & rj) == 0) {
                        const unsigned long long x = v[r], y = v[r | rj];
                        v[r] = umin64(x, y);
                        v[r | rj] = umax64(x, y);
                    }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const unsigned long long p = __shfl_xor_sync(0xffffffffu, v[r], j);
                    v[r] = lower ? umin64(v[r], p) : umax64(v[r], p);
                }
            }
        }
    }
}

template <int N>
__device__ __forceinline__ void warp_sort_list(const uint32_t *__restrict__ bkey, const uint32_t *__restrict__ bval,
                                               int64_t lo, int L, uint32_t t, uint32_t *skey, uint32_t *sval, int lane)
{
    unsigned long long v[N / 32];
#pragma unroll
    for (int r = 0; r < N / 32; r++) {
        const int e = r * 32 + lane;
        v[r] = e < L ? ((unsigned long long)bkey[lo + e] << 32 | bval[lo + e]) : ~0ull;
    }
    warp_bitonic<N>(v, lane);
#pragma unroll
    for (int r = 0; r < N / 32; r++) {
        const int e = r * 32 + lane;
        if (e < L) {
            skey[lo + e] = t;
            sval[lo + e] = (uint32_t)v[r];
        }
    }
}

constexpr int SORT_WARP_MAX = LONG_LIST; // lists up to this length: one warp, in registers
constexpr int SORT_SMEM_MAX = 2048;      // longer ones up to this: one block, in shared memory (16 KB)

// The tiles whose lists have more than SORT_WARP_MAX keys (for
// k_tile_sort_long) and more than FIRST_LIST keys (for the rasterizers to take
// first), from the scanned list offsets.
__global__ void k_find_long(const uint32_t *__restrict__ tile_off, int tiles, int64_t kcap, int *n_long,
                            int32_t *long_tiles, int *n_first, int32_t *first_tiles)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
        const int64_t lo = min((int64_t)tile_off[t], kcap), hi = min((int64_t)tile_off[t + 1], kcap);
        const int L = (int)(hi - lo);
        if (L > SORT_WARP_MAX) long_tiles[atomicAdd(n_long, 1)] = t;
        if (L > FIRST_LIST) first_tiles[atomicAdd(n_first, 1)] = t;
    }
}

// One warp per tile: the tile's range, and its list sorted into (tile, splat)
// order when it has at most SORT_WARP_MAX keys (longer lists are
// k_tile_sort_long's).
__global__ void __launch_bounds__(256) k_tile_sort(const uint32_t *__restrict__ tile_off, int tiles, int64_t kcap,
                                                   const uint32_t *__restrict__ bkey,
                                                   const uint32_t *__restrict__ bval, uint32_t *skey, uint32_t *sval,
                                                   uint2 *ranges)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tiles; t += nwarps) {
        const int64_t lo = min((int64_t)tile_off[t], kcap), hi = min((int64_t)tile_off[t + 1], kcap);
        const int L = (int)(hi - lo);
        if (lane == 0) ranges[t] = make_uint2((uint32_t)lo, (uint32_t)hi);
        if (L <= 0) continue;
        if (L <= 32) warp_sort_list<32>(bkey, bval, lo, L, (uint32_t)t, skey, sval, lane);
        else if (L <= 64) warp_sort_list<64>(bkey, bval, lo, L, (uint32_t)t, skey, sval, lane);
        else if (L <= 128) warp_sort_list<128>(bkey, bval, lo, L, (uint32_t)t, skey, sval, lane);
        else if (L <= SORT_WARP_MAX) warp_sort_list<256>(bkey, bval, lo, L, (uint32_t)t, skey, sval, lane);
    }
}

// Compare-exchange of positions i < j of a list of length L (positions >= L
// hold +inf and stay untouched).
__device__ __forceinline__ void cmpx_smem(unsigned long long *v, int i, int j)
{
    const unsigned long long x = v[i], y = v[j];
    if (y < x) {
        v[i] = y;
        v[j] = x;
    }
}
__device__ __forceinline__ void cmpx_global(uint32_t *key, uint32_t *val, int64_t lo, int L, int i, int j)
{
    if (j >= L) return;
    const unsigned long long x = (unsigned long long)key[lo + i] << 32 | val[lo + i];
    const unsigned long long y = (unsigned long long)key[lo + j] << 32 | val[lo + j];
    if (y < x) {
        key[lo + i] = (uint32_t)(y >> 32);
        val[lo + i] = (uint32_t)y;
        key[lo + j] = (uint32_t)(x >> 32);
        val[lo + j] = (uint32_t)x;
    }
}

// One block per long list: a bitonic sort in shared memory (up to
// SORT_SMEM_MAX keys, padded to a power of two with +inf), else in place in
// the unsorted key arrays (positions past the list act as +inf).
__global__ void __launch_bounds__(256) k_tile_sort_long(const uint32_t *__restrict__ tile_off, int64_t kcap,
                                                        uint32_t *bkey, uint32_t *bval, uint32_t *skey,
                                                        uint32_t *sval, const int *n_long,
                                                        const int32_t *__restrict__ long_tiles)
{
    extern __shared__ unsigned long long sv[];
    const int nl = *n_long;
    for (int q = blockIdx.x; q < nl; q += gridDim.x) {
        const int t = long_tiles[q];
        const int64_t lo = min((int64_t)tile_off[t], kcap), hi = min((int64_t)tile_off[t + 1], kcap);
        const int64_t L64 = hi - lo;
        if (L64 > (1 << 30)) continue;                   // beyond any workspace; the list stays unsorted
        const int L = (int)L64;
        int P = 1;
        while (P < L) P <<= 1;
        const bool in_smem = P <= SORT_SMEM_MAX;
        if (in_smem)
            for (int e = threadIdx.x; e < P; e += blockDim.x)
                sv[e] = e < L ? ((unsigned long long)bkey[lo + e] << 32 | bval[lo + e]) : ~0ull;
        __syncthreads();
        for (int lk = 1; (1 << lk) <= P; lk++) {        // blocks of k = 2^lk
            const int k = 1 << lk;
            for (int e = threadIdx.x; e < P / 2; e += blockDim.x) {      // mirrored pairs within blocks of k
                const int i = ((e >> (lk - 1)) << lk) | (e & ((k >> 1) - 1)), j = i ^ (k - 1);
                if (in_smem) cmpx_smem(sv, i, j);
                else cmpx_global(bkey, bval, lo, L, i, j);
            }
            __syncthreads();
            for (int ld = lk - 2; ld >= 0; ld--) {       // then pairs at distance 2^ld
                for (int e = threadIdx.x; e < P / 2; e += blockDim.x) {
                    const int i = ((e >> ld) << (ld + 1)) | (e & ((1 << ld) - 1)), j = i + (1 << ld);
                    if (in_smem) cmpx_smem(sv, i, j);
                    else cmpx_global(bkey, bval, lo, L, i, j);
                }
                __syncthreads();
            }
        }
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            skey[lo + e] = (uint32_t)t;
            sval[lo + e] = in_smem ? (uint32_t)sv[e] : bval[lo + e];
        }
        __syncthreads();                                  // sv is reused by the next list
    }
}

// Counts, scan, emission and per-tile sorts of one view's lists, from the
// records, rectangles, depths and big list the gather left in rb.
void build_tile_lists(const DevArgs *args, int view, const int *n_vis, RenderBufs &rb, int tiles, Work &w,
                      cudaStream_t s)
{
    const int cap = (int)rb.cap;
    cudaMemsetAsync(rb.tile_cnt, 0, (size_t)(tiles + 1) * sizeof(uint32_t), s);
    cudaMemsetAsync(rb.tile_cur, 0, (size_t)tiles * sizeof(uint32_t), s);
    // the key count of every tile
    const int gsm = w.grid((int64_t)(cap + 31) / 32 * 32, TILES_BLOCK);
    k_tiles_count<<<gsm, TILES_BLOCK, 0, s>>>(rb.rect, rb.rec0, rb.rec1, rb.fix_flag, n_vis, cap, args, view,
                                              rb.tile_cnt, rb.reach);
    w.wait_side(s);                                       // the FP64 fix-ups (prepare_view) have landed
    k_big_counts<<<w.num_sms * 4, 256, 0, s>>>(rb.rec0, rb.rec1, rb.rect, rb.n_big, rb.big_idx, cap, args, view,
                                               rb.tile_cnt);
    // each tile's first key (and the key total), then the keys into their tiles' lists
    scan_counts(rb.tile_cnt, tiles + 1, rb.n_keys, (int)rb.kcap, w, s);
    k_tiles_emit<<<gsm, TILES_BLOCK, 0, s>>>(rb.rect, rb.reach, rb.depth, n_vis, cap, rb.kcap, args, view, rb.tile_cnt,
                                             rb.tile_cur, rb.tk[0], rb.tv[0]);
    k_big_emit<<<w.num_sms * 4, 256, 0, s>>>(rb.rect, rb.rec0, rb.rec1, rb.depth, rb.n_big, rb.big_idx, cap, rb.kcap,
                                             args, view, rb.tile_cnt, rb.tile_cur, rb.tk[0], rb.tv[0]);
    // front-to-back order within each tile, and the tiles' ranges: the long
    // lists (a block each) on the side stream beside the others (a warp each)
    k_find_long<<<w.grid(tiles, 256, 2), 256, 0, s>>>(rb.tile_cnt, tiles, rb.kcap, rb.n_big + 1, rb.long_tiles,
                                                       rb.n_big + 2, rb.first_tiles);
    static_assert(SORT_SMEM_MAX * sizeof(unsigned long long) <= 48 * 1024,
                  "the long-list buffer stays within the default dynamic shared-memory limit");
    const cudaStream_t fs = w.fork(s);
    k_tile_sort_long<<<w.num_sms * 6, 256, SORT_SMEM_MAX * sizeof(unsigned long long), fs>>>(
        rb.tile_cnt, rb.kcap, rb.tk[0], rb.tv[0], rb.tk[1], rb.tv[1], rb.n_big + 1, rb.long_tiles);
    w.side_done(fs);
    k_tile_sort<<<w.grid((int64_t)tiles * 32, 256), 256, 0, s>>>(rb.tile_cnt, tiles, rb.kcap, rb.tk[0], rb.tv[0],
                                                                  rb.tk[1], rb.tv[1], rb.ranges);
    w.wait_side(s);
}

}  // namespace gs
