// gs_kernels.cuh -- host-side launchers of the hot-path kernels and the
// scratch-workspace view they share.
#pragma once

#include <type_traits>

#include "gs_internal.cuh"

namespace gs {

// Length of a scan: fixed, or mul * ceil(min(*n_dev, cap) / div) + add.
struct ScanLen {
    const int *n_dev;
    int mul, div, add, fixed, cap;
};

// Polls of an mbarrier before a wait on the block's own TMA copies gives up
// (the block then latches GS_ERR_TIMEOUT, lets its copies land and returns).
constexpr uint32_t CULL_WAIT_LIMIT = 1u << 24;

struct Work {
    uint32_t *partials;   // >= 1024 scan partials (and 1024 more after them for work on the side stream)
    int *status;          // device status word
    int scan_grid;        // blocks of the scan kernels (<= 1024)
    int num_sms;
    cudaEvent_t *tev;     // timing points of the current step, or nullptr
    bool capturing;       // the stream is being captured into a graph
    uint32_t cull_first_wait = CULL_WAIT_LIMIT;   // limit of each cull block's first wait (failure-path tests)
    // A second stream for short independent kernels (the FP64 fix-ups) that
    // run beside the main stream's work: fork() returns the stream to launch
    // on, side_done() marks the end of that work, wait_side() makes the main
    // stream wait for it.  Without a side stream everything stays on s.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t fork(cudaStream_t s) const
    {
        if (!side) return s;
        cudaEventRecord(ev_fork, s);
        cudaStreamWaitEvent(side, ev_fork, 0);
        return side;
    }
    void side_done(cudaStream_t fs) const
    {
        if (side && fs == side) cudaEventRecord(ev_join, side);
    }
    void wait_side(cudaStream_t s) const
    {
        if (side) cudaStreamWaitEvent(s, ev_join, 0);
    }
    void mark(int p, cudaStream_t s) const
    {
        if (!tev) return;
        // External: recorded as an event node when the stream is being captured
        if (capturing) cudaEventRecordWithFlags(tev[p], s, cudaEventRecordExternal);
        else cudaEventRecord(tev[p], s);
    }
    int grid(int64_t threads, int block, int per_sm = 8) const
    {
        int64_t b = (threads + block - 1) / block;
        int64_t mx = (int64_t)num_sms * per_sm;
        if (b > mx) b = mx;
        return (int)(b < 1 ? 1 : b);
    }
};

// k_scan.cu
void scan_exclusive(const uint32_t *in, uint32_t *out, ScanLen L, Work &w, int *total_out, int total_cap,
                    cudaStream_t s);
// Exclusive scan of len counts in place (one block when len <= 65536, else
// scan_exclusive); the total goes to total_out, clamped to cap with
// GS_ERR_CAPACITY latched above it.
void scan_counts(uint32_t *v, int64_t len, int *total_out, int cap, Work &w, cudaStream_t s);
// dst[k * planes + r] = src[r * spitch + k] for k < min(*n, cap), r < planes.
void launch_to_rows(const float *src, int64_t spitch, int planes, const int *n, int cap, float *dst, Work &w,
                    cudaStream_t s);
// dst[k] = src[ids[k]] for k < min(*n, cap).
void launch_gather_u8(const uint8_t *src, const int32_t *ids, const int *n, int cap, uint8_t *dst, Work &w,
                      cudaStream_t s);
void compact_mask(const uint32_t *mask, int64_t n, uint32_t *chunk_cnt, bool have_counts, int32_t *ids,
                  uint32_t *word_prefix, int cap, int *count_out, Work &w, cudaStream_t s, uint8_t *counter = nullptr,
                  uint8_t *delay = nullptr);

// SH planes of w, m, v and their restore directions: D - 11 planes each, of
// the SH storage type.  Resident scenes: the planes sit `ppitch` = pitch
// elements apart inside the scene's arrays and Gaussian i at element i.  Host
// tier: they sit in the context's staging ring, ppitch = slots << shift, and
// Gaussian i at (slot[i >> shift] << shift) + (i & (2^shift - 1)).
struct ShRows {
    void *w, *m, *v, *rdir;   // rdir may be nullptr (then restores use m, v)
    int64_t ppitch;
    const int32_t *slot;      // host tier: chunk -> staging slot; nullptr when resident
    int shift;
    // Forwarded rows (GS_TIER_HOST_CPU_OPT): w holds the current SH values of
    // the step's visible Gaussians (no restore, m and v absent), Gaussian i at
    // its rank in the visibility mask cmask (word prefix cprefix).
    const uint32_t *cmask, *cprefix;
    int current;
    __device__ __forceinline__ int64_t base(int64_t i) const
    {
        if (cmask)
            return (int64_t)__ldg(cprefix + (i >> 5)) + __popc(__ldg(cmask + (i >> 5)) & ((1u << (i & 31)) - 1u));
        if (!slot) return i;
        // a chunk the step did not stage has slot -1: never read for a staged
        // step's Gaussians; clamped so a stray index stays inside the ring
        return ((int64_t)max(__ldg(slot + (i >> shift)), 0) << shift) + (i & ((1ll << shift) - 1));
    }
};

// Scene pointers as the kernels take them.
struct SceneView {
    float *geo;           // [11][pitch] fp32
    void *m;              // geometry rows of m: [11][pitch], fp32 or bf16 (prec); SH rows in sh
    void *v;
    float *rdir;          // [11][pitch] fp32 geometry restore directions, or nullptr
    ShRows sh;
    uint8_t *counter;
    int64_t n, pitch;
    int deg, D;
    int prec;             // GS_FP32, GS_BF16_SH_MOM or GS_BF16_SH_MOM_RN
    int tier;             // GS_TIER_DEVICE or GS_TIER_HOST_SH
    int opt;              // optimizer whose state the planes hold (GS_OPT_*): picks the restoring kernels
};

// Calls f(std::integral_constant<int, GS_OPT_x>{}) for the optimizer kind
// `opt`, so a launcher instantiates its kernel per kind.  Host only.
template <class F> inline void with_opt(int opt, F &&f)
{
    switch (opt) {
    case GS_OPT_ADAMW: f(std::integral_constant<int, GS_OPT_ADAMW>{}); break;
    case GS_OPT_SGDM: f(std::integral_constant<int, GS_OPT_SGDM>{}); break;
    default: f(std::integral_constant<int, GS_OPT_ADAM>{}); break;
    }
}

// Timing points recorded inside a step (see gs_timing_enable).
enum { TP_STEP0 = 0, TP_CULL0, TP_CULL1, TP_FWD0, TP_FWD1, TP_BWD0, TP_BWD1, TP_ADAM0, TP_APPLY0, TP_APPLY1,
       TP_ADAM1, TP_STEP1, TP_RBWD0, TP_RBWD1, TP_COUNT };

// gs_runtime.cu: the Adam hyper-parameters are usable (betas in [0, 1), eps >= 0,
// max_defer in [1, 15], a known mode).  Host only.
bool valid_adam(const gs_adam_cfg *a);
// gs_noalloc.cu: the first-wait limit of gs_cull_noalloc's cull blocks.
void set_noalloc_first_wait(uint32_t limit);

// k_cull.cu: visibility bitmask + per-chunk counts (restore if lut.restore).
void launch_cull(const SceneView &sc, const DevArgs *args, int view, uint32_t *mask, uint32_t *chunk_cnt, Work &w,
                 cudaStream_t s);
// All views of a step in one sweep over the geometry (per-view masks and chunk counts).
// With umask, the same sweep also takes the deferred optimizer's select
// (returns true; false if it fell back to per-view sweeps without it).
// n_cand (optional) receives the number of Gaussians that passed the
// pre-test in some view (their rotation planes were read).
bool launch_cull_views(const SceneView &sc, const DevArgs *args, int n_views, uint32_t *const *masks,
                       uint32_t *const *chunk_cnts, Work &w, cudaStream_t s, uint32_t *umask = nullptr,
                       uint32_t *uchunk = nullptr, int max_defer = 0, int *n_cand = nullptr);
void launch_ids_to_mask(const int32_t *ids, const int *n_dev, int cap, uint32_t *mask, int64_t n, Work &w,
                        cudaStream_t s);
void launch_mask_or(uint32_t *dst, const uint32_t *src, int64_t nwords, Work &w, cudaStream_t s);

// k_adam.cu
struct PairBufs;
// Select, then the pair-wise apply when pb is given and the scene allows it,
// else the member-wise compaction and apply.
void launch_adam_deferred(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                          const float *grad, int64_t gcap, uint32_t *umask, uint32_t *uchunk, int32_t *uids,
                          uint8_t *udelay, int *n_upd, Work &w, cudaStream_t s, const PairBufs *pb = nullptr);
void launch_adam_eager(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, Work &w, cudaStream_t s);
void launch_adam_select(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, uint32_t *umask,
                        uint32_t *uchunk, int32_t *uids, uint8_t *udelay, int *n_upd, Work &w, cudaStream_t s);
void launch_adam_apply(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, const int32_t *uids, const uint8_t *udelay,
                       const int *u_range, const int *n_upd, Work &w, cudaStream_t s);
void launch_adam_compact(const SceneView &sc, uint32_t *umask, uint32_t *uchunk, int32_t *uids, uint8_t *udelay,
                         int *n_upd, Work &w, cudaStream_t s);
// The pair-wise apply (resident scenes): update set taken as Gaussian pairs.
struct PairBufs {
    uint32_t *pmask;      // [n/64 + CHUNK_WORDS] pairs with a member
    uint32_t *pchunk;     // [n/4096 + 1] per-chunk counts
    int32_t *pids;        // [n/2 + 1] active pairs, ascending
    uint32_t *pinfo;      // [n/2 + 1] delays and member bits of each
    int *n_pairs;         // device count
};
bool adam_pairs_ok(const SceneView &sc);
// After the select (update-set mask and per-chunk member counts): the member
// count to n_upd, the active pairs, their delays (members' counters cleared)
// and the apply.
void launch_adam_pairs(const SceneView &sc, const DevArgs *args, const uint32_t *vmask, const uint32_t *vprefix,
                       const float *grad, int64_t gcap, uint32_t *umask, uint32_t *uchunk, const PairBufs &pb,
                       int *n_upd, Work &w, cudaStream_t s);
// The same in two parts: the pairs and their delays, which need only the
// select (and can run beside the render), with the counters left as they are;
// then the apply, which clears the members' counters.
void launch_adam_pairs_prep(const SceneView &sc, uint32_t *umask, uint32_t *uchunk, const PairBufs &pb, int *n_upd,
                            Work &w, cudaStream_t s);
void launch_adam_pairs_apply(const SceneView &sc, const DevArgs *args, const uint32_t *vmask,
                             const uint32_t *vprefix, const float *grad, int64_t gcap, const PairBufs &pb, Work &w,
                             cudaStream_t s);
void launch_touch_from_masks(const uint32_t *vmask, const uint32_t *umask, int64_t n, int shift, uint8_t *touch,
                             Work &w, cudaStream_t s);
void launch_uid_range(const int32_t *uids, const int *n_upd, int64_t id_lo, int64_t id_hi, int *range, cudaStream_t s);
void launch_touch_chunks(const uint32_t *vmask, const uint8_t *counter, int64_t n, int shift, int max_defer,
                         uint8_t *touch, Work &w, cudaStream_t s);
// Device camera of a view: pinhole, the projection's guard band, the camera
// centre and the tile grid.  Host only.
DevCam make_cam(const gs_camera &a, int tile_w, int tile_h);
// A camera's region fields describe a whole image or a region inside its full image.
bool camera_region_ok(const gs_camera &a);
// Deferred-update tables (Fig. 10) for optimizer step t; restore = 0 leaves the
// cull's and gather's restore off.  Host only.
DevLut make_lut(const gs_adam_cfg *a, int t, bool restore, int precision = GS_FP32);
void launch_refresh_rdir(const SceneView &sc, const DevArgs *args, Work &w, cudaStream_t s);
void launch_materialize(const SceneView &sc, const DevArgs *args, float *w_out, float *m_out, float *v_out,
                        Work &w, cudaStream_t s);
void launch_grad_scatter(const int32_t *ids, const int *n_dev, int cap, const float *gc, int64_t gcap, int D,
                         float *gfull, int64_t pitch, Work &w, cudaStream_t s);

// k_densify.cu: clone / split / prune on deferred state.  densify_count
// classifies every Gaussian (masks[0..2]: survivor, clone, split; their word
// prefixes and counts); densify_write writes the new scene's rows.
gs_status densify_count(const SceneView &sc, const DevArgs *args, const float *accum, const float *denom,
                        float grad_threshold, float scale_limit, float min_opacity, uint32_t *const masks[3],
                        uint32_t *const prefixes[3], uint32_t *const chunks[3], int *counts, Work &w, cudaStream_t s);
void densify_write(const SceneView &sc, const SceneView &dst, const DevArgs *args, const float *normals,
                   uint32_t *const masks[3], uint32_t *const prefixes[3], const int *counts, Work &w, cudaStream_t s);

// k_render.cu
// Per-splat record of the rasterizer backward's sums: d/d(mean2d x, y), d/d(conic
// A, B, C), d/d(opacity), d/d(rgb), padded to 12 floats so that a warp adds
// them with two 16-byte vector atomics and one scalar.
constexpr int G9_STRIDE = 12;

struct RenderBufs {
    float *compact;          // [D][cap] restored parameters of the visible set
    int64_t cap;             // visible capacity
    float4 *rec0, *rec1, *rec2;
    uint2 *rect;
    uint32_t *depth;         // [cap] depth of each visible splat (f32 bits: positive, so ordered as integers)
    uint32_t *tile_cnt;      // [tiles + 1] keys per tile, then (scanned in place) each tile's first key
    uint32_t *tile_cur;      // [tiles] emission cursors
    int32_t *long_tiles;     // [tiles] tiles whose lists are sorted by k_tile_sort_long
    int32_t *first_tiles;    // [tiles] tiles with more than FIRST_LIST keys (rasterized first)
    uint32_t *tk[2], *tv[2]; // keys: [0] per tile, unsorted (depth, splat); [1] sorted (tile, splat)
    int64_t kcap;            // key capacity
    uint2 *ranges;           // [tiles]
    float *g9;               // [cap][G9_STRIDE] per splat, summed over its pixels (ds = -alpha dL/dalpha):
                             // ds dx, ds dy, ds dx^2, ds dx dy, ds dy^2, ds, dL/d rgb (9 used)
    int *n_keys;             // device
    float *cfinal;           // [3][H][W] final colour of the last forward render (for the backward)
    int *n_fix;              // device: Gaussians handed to the FP64 fix-up passes
    int32_t *fix_idx;        // [cap] their visible-set indices
    uint8_t *fix_flag;       // [cap] 1 for those, else 0
    int *n_big;              // device [3]: [0] splats of the large-rectangle list, [1] long tiles, [2] first tiles
    float4 *lrec;            // [3 kcap] splat records in list order (rec0, rec1, rec2 with rec2.w = splat index
                             // bits), written for the TMA-staged rasterizer variant
    int32_t *big_idx;        // [cap] splats whose tiles a warp counts and emits (k_big_counts, k_big_emit)
    uint32_t *reach;         // [cap] small-rectangle splats: bit j set when the j-th tile of the rectangle
                             // (row-major) is reached (written by the key count, read by the emission)
    int variant;             // forward rasterizer variant (pixels per thread, batch), see raster_variant_ok
    int variant_bwd;         // backward rasterizer variant
    // filled by render_fwd
    const uint32_t *sorted_keys;
    const uint32_t *sorted_vals;
    int tiles;
};

// The rasterizer's work over one or several views: (view, tile) items
// [tile_ofs[v], tile_ofs[v + 1]) are view v's tiles; persistent blocks take
// items from a work counter (zeroed before each launch) until all are done,
// each view's long lists first (so that none of them starts late and leaves
// the GPU to a few warps at the end), then its other tiles in order.
struct RasterJob {
    int n_views;
    int tile_ofs[MAX_VIEWS + 1];
    const uint2 *ranges[MAX_VIEWS];
    const uint32_t *svals[MAX_VIEWS];
    const float4 *rec0[MAX_VIEWS], *rec1[MAX_VIEWS], *rec2[MAX_VIEWS];
    float *image[MAX_VIEWS];     // forward: image out
    float *cfinal[MAX_VIEWS];    // forward: final colour kept for the backward (or null); backward: read
    float *dimage[MAX_VIEWS];    // forward: dL/dimage out (with targets); backward: read
    float *g9[MAX_VIEWS];        // backward: per-splat sums out
    uint32_t cap[MAX_VIEWS];     // visible capacity (list entries index records below it)
    const float4 *lrec[MAX_VIEWS];   // records in list order (TMA-staged variant)
    const int32_t *first_tiles[MAX_VIEWS];  // tiles whose lists exceed FIRST_LIST keys (k_tile_sort)
    const int *n_first[MAX_VIEWS];           // device: their number (null: none)
    int *status;                 // device status word (a TMA wait that gave up)
    uint32_t first_wait;         // polls of each warp's first TMA wait (CULL_WAIT_LIMIT unless a test lowers it)
    int cam0;                    // job view v is camera cam0 + v of the argument block
    int *work;
};

// Lists longer than LONG_LIST are sorted by a block (k_tile_sort_long); lists
// longer than FIRST_LIST (about three times the mean of a dense 8x4-tile
// view; 64, 96, 160, 192 and 256 measured slower on the 10M aerial step) are
// handed to the rasterizers before the others.
constexpr int LONG_LIST = 256;
constexpr int FIRST_LIST = 128;

constexpr int N_RASTER_VARIANTS = 10;
// The variant whose lists are staged by TMA bulk copies from records in list order.
constexpr int RASTER_TMA_VARIANT = 9;

// k_lists.cu: rectangles of more tiles than this are counted and emitted by a
// warp each (the big list the gather fills); smaller ones by a warp's lanes
// over the concatenated (splat, tile) pairs of 32 splats.
constexpr int BIG_RECT = 32;
void build_tile_lists(const DevArgs *args, int view, const int *n_vis, RenderBufs &rb, int tiles, Work &w,
                      cudaStream_t s);
// has_records: the context keeps list-order records (variant 9 needs them).
bool raster_variant_ok(int v, int tile_w, int tile_h, bool has_records);

void render_forward(const SceneView &sc, const DevArgs *args, int view, const int32_t *ids, const int *n_vis,
                    RenderBufs &rb, const DevCam &cam_host, float *image, bool use_target, float *dimage,
                    float *loss, Work &w, cudaStream_t s, int *work);
// The stages of render_forward / render_backward, for steps over several views:
// per view prepare_view (gather, projection, keys, sorts); one forward and one
// backward rasterizer launch over all views; per view project_backward.
// zero_g9: also clear the view's per-splat gradient sums (on the side stream,
// beside the list building), for a raster_backward told g9_zeroed.
void prepare_view(const SceneView &sc, const DevArgs *args, int view, const int32_t *ids, const int *n_vis,
                  RenderBufs &rb, const DevCam &cam_host, Work &w, cudaStream_t s, bool zero_g9 = false);
// cam0: the job's views are cameras cam0.. of the argument block (a round of
// a step's views); rbs, images, dimages and n_vis are per job view.
void raster_forward(const DevArgs *args, int n_views, RenderBufs *const *rbs, const DevCam *cams, float *const *images,
                    bool use_target, float *const *dimages, float *loss, int *work, Work &w, cudaStream_t s,
                    int cam0 = 0);
void raster_backward(const DevArgs *args, int n_views, RenderBufs *const *rbs, const DevCam *cams,
                     const float *const *dimages, const int *const *n_vis, int *work, Work &w, cudaStream_t s,
                     unsigned long long *stats = nullptr, int cam0 = 0, bool g9_zeroed = false);
// Visibility masks of the views rendered before this one in a step over
// several views.  A Gaussian that none of them sees takes its gradient row by
// plain stores (so the union layout needs no zeroing first); the others add.
struct PrevMasks {
    const uint32_t *m[MAX_VIEWS];
    int n;
};
void project_backward(const SceneView &sc, const DevArgs *args, int view, const int *n_vis, RenderBufs &rb,
                      float *grad, int64_t gcap, const uint32_t *remap_mask, const uint32_t *remap_prefix,
                      const int32_t *ids, const PrevMasks &prev, Work &w, cudaStream_t s);
void render_backward(const SceneView &sc, const DevArgs *args, int view, const int *n_vis, RenderBufs &rb,
                     const DevCam &cam_host, const float *dimage, float *grad, int64_t gcap,
                     const uint32_t *remap_mask, const uint32_t *remap_prefix, const int32_t *ids,
                     Work &w, cudaStream_t s, int *work, unsigned long long *stats = nullptr);
void launch_loss_l1(const float *image, const float *target, int64_t count, float *loss, float *dimage, Work &w,
                    cudaStream_t s);
void launch_zero_rows(float *buf, int rows, int64_t pitch, const int *n_dev, int cap, Work &w, cudaStream_t s,
                      bool aos = false);

}  // namespace gs
